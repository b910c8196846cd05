// yee_step_cell.cuh -- the whole Yee step in one cell-parallel kernel (sm_103a).
//
// One thread per cell (i, j, k) does rows a2-a6 of a step for its cell:
//   * H^{n+1/2} of its own cell (curl of E^n, CPML psi of the H side, soft
//     source at (n+1/2) dt; Section 4, Eq. 13b), stored;
//   * H^{n+1/2} of the nine neighbouring components the rest needs,
//     recomputed in registers and not stored: Hy, Hz at i-1; Hx, Hz at j-1;
//     Hx, Hy at k-1 (the E curl) and Hx at i+1, Hy at j+1, Hz at k+1 (the
//     cell-centred H-bar of the fluence);
//   * E^{n+1} of its own cell (curl of H^{n+1/2}, CPML psi of the E side,
//     PEC walls, soft source at (n+1) dt; Eq. 13a), stored;
//   * the fluence term |E^n_c x Hbar^n_c| dt of its cell (Section 2).
// The step therefore reads E^n, H^{n-1/2} and the fluence once and writes
// E^{n+1}, H^{n+1/2} and the fluence once -- the least traffic of a step --
// with no shared memory, no barrier and no z loop: the +-1 neighbours come
// through L1 / L2 from the loads of adjacent threads and of the blocks of
// the neighbouring planes, which run at about the same time.  The H-side psi
// is read from the read copy and written to the write copy, so recomputing
// a neighbour's H races with nobody; the E-side psi of a cell is touched by
// its own thread only.
//
// Blocks whose cells or +-1 neighbours reach a wall, a ragged edge or the
// CPML shell compile every check in (GEN); the others none.  Bit 6 of the
// column mask (set on the host) marks columns whose own or +-x / +-y
// neighbour column carries an H antenna point; only those cells evaluate
// source terms of recomputed neighbours.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "yee_cell.cuh"

namespace fdtd {

template <typename real, bool GEN>
struct CellNbhd {
    const StepArgs<real>& a;
    int i, j, k;       // own cell
    int g;             // own linear index
    int zp, zm;        // offsets of planes k+1, k-1 from plane k (z wraps)
    int kp, km;        // wrapped plane indices k+1, k-1
    Cpx<real> th;      // f e^{-i Phi} at the H time

    __device__ __forceinline__ bool in(int di, int dj) const
    {
        return !GEN || (i + di >= 0 && i + di < a.nx && j + dj >= 0 && j + dj < a.ny);
    }
    __device__ __forceinline__ int off(int di, int dj, int dz) const
    {
        return di + dj * a.pitch + (dz > 0 ? zp : (dz < 0 ? zm : 0));
    }
    __device__ __forceinline__ real E(int c, int di, int dj, int dz) const
    {
        return in(di, dj) ? __ldg(a.ein[c] + g + off(di, dj, dz)) : real(0);
    }
    __device__ __forceinline__ real Ho(int c, int di, int dj, int dz) const
    {
        return in(di, dj) ? __ldg(a.hin[c] + g + off(di, dj, dz)) : real(0);
    }
    __device__ __forceinline__ int plane_of(int dz) const { return dz > 0 ? kp : (dz < 0 ? km : k); }

    // H^{n+1/2} component C of the cell at (i+DI, j+DJ, k+DZ); zero outside
    // the grid.  `store` writes the psi of the H side (own cell only).
    template <int C, int DI, int DJ, int DZ>
    __device__ __forceinline__ real H(bool src, bool store = false) const
    {
        if (!in(DI, DJ)) return real(0);
        const int ci = i + DI, cj = j + DJ, ck = plane_of(DZ);
        real h = Ho(C, DI, DJ, DZ);
        real d1, d2;   // the two differences of the curl
        if (C == 0) {
            d1 = E(2, DI, DJ + 1, DZ) - E(2, DI, DJ, DZ);    // dEz/dy
            d2 = E(1, DI, DJ, DZ + 1) - E(1, DI, DJ, DZ);    // dEy/dz
            h = h - __ldg(a.chy + cj) * d1 + a.cz * d2;
        } else if (C == 1) {
            d1 = E(2, DI + 1, DJ, DZ) - E(2, DI, DJ, DZ);    // dEz/dx
            d2 = E(0, DI, DJ, DZ + 1) - E(0, DI, DJ, DZ);    // dEx/dz
            h = h - a.cz * d2 + __ldg(a.chx + ci) * d1;
        } else {
            d1 = E(1, DI + 1, DJ, DZ) - E(1, DI, DJ, DZ);    // dEy/dx
            d2 = E(0, DI, DJ + 1, DZ) - E(0, DI, DJ, DZ);    // dEx/dy
            h = h - __ldg(a.chx + ci) * d1 + __ldg(a.chy + cj) * d2;
        }
        if (GEN && a.npml > 0) {
            const int npml = a.npml, w2 = 2 * npml, nx = a.nx, ny = a.ny;
            if (C != 0 && (ci < npml || ci >= nx - npml)) {   // x shell: Hyx (d1 = dEz/dx), Hzx (d1 = dEy/dx)
                const int ii = ci < npml ? ci : ci - nx + w2;
                const int q = (ck * ny + cj) * w2 + ii;
                const real p = a.bhx[ii] * a.phx_in[C - 1][q] + a.ahx[ii] * d1;
                if (C == 1) h += p; else h -= p;
                if (store) a.phx_out[C - 1][q] = p;
            }
            if (C != 1 && (cj < npml || cj >= ny - npml)) {   // y shell: Hxy (d1 = dEz/dy), Hzy (d2 = dEx/dy)
                const int jj = cj < npml ? cj : cj - ny + w2;
                const int q = (ck * w2 + jj) * a.pitch + ci;
                const int slot = C == 0 ? 0 : 1;
                const real p = a.bhy[jj] * a.phy_in[slot][q] + a.ahy[jj] * (C == 0 ? d1 : d2);
                if (C == 0) h -= p; else h += p;
                if (store) a.phy_out[slot][q] = p;
            }
        }
        if (src && a.smask) {
            const int col = cj * a.nx + ci;
            if (__ldg(a.smask + col) & (0x08 << C)) h += src_add(a, 3 + C, col, plane_factor(a, ck, th));
        }
        return h;
    }
};

template <typename real, bool GEN>
__device__ __forceinline__ void step_cell(const StepArgs<real>& a, const StepTime<real>& t, int i, int j, int k)
{
    using Acc = FluAcc<real>;
    using acc_t = typename Acc::T;
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    if (GEN && (i >= nx || j >= ny)) return;
    const int plane = pitch * ny;
    CellNbhd<real, GEN> N{a, i, j, k, k * plane + j * pitch + i, 0, 0, 0, 0, t.th};
    N.kp = k + 1 == nz ? 0 : k + 1;
    N.km = k == 0 ? nz - 1 : k - 1;
    N.zp = (N.kp - k) * plane;
    N.zm = (N.km - k) * plane;
    const int g = N.g, col = j * nx + i;
    const uint8_t mk = a.smask ? __ldg(a.smask + col) : uint8_t(0);
    const bool hsrc = (mk & 0x40) != 0;   // an H antenna point in this or a +-x / +-y column

    // ---- H^{n+1/2}: own (stored) and the neighbours the E curl and H-bar need
    const real hx = N.template H<0, 0, 0, 0>(hsrc, true);
    const real hy = N.template H<1, 0, 0, 0>(hsrc, true);
    const real hz = N.template H<2, 0, 0, 0>(hsrc, true);
    a.hout[0][g] = hx; a.hout[1][g] = hy; a.hout[2][g] = hz;
    const real hy_im = N.template H<1, -1, 0, 0>(hsrc);
    const real hz_im = N.template H<2, -1, 0, 0>(hsrc);
    const real hx_jm = N.template H<0, 0, -1, 0>(hsrc);
    const real hz_jm = N.template H<2, 0, -1, 0>(hsrc);
    const real hx_km = N.template H<0, 0, 0, -1>(hsrc);
    const real hy_km = N.template H<1, 0, 0, -1>(hsrc);

    // ---- E^{n+1} of the own cell
    const real ex = N.E(0, 0, 0, 0), ey = N.E(1, 0, 0, 0), ez = N.E(2, 0, 0, 0);
    const real cex = __ldg(a.cex + i), cey = __ldg(a.cey + j), cz = a.cz;
    const real dHz_y = hz - hz_jm, dHy_z = hy - hy_km, dHx_z = hx - hx_km;
    const real dHz_x = hz - hz_im, dHy_x = hy - hy_im, dHx_y = hx - hx_jm;
    real nex = ex + cey * dHz_y - cz * dHy_z;
    real ney = ey + cz * dHx_z - cex * dHz_x;
    real nez = ez + cex * dHy_x - cey * dHx_y;
    if (GEN && a.npml > 0) {
        const int npml = a.npml, w2 = 2 * npml;
        if (i < npml || i >= nx - npml) {
            const int ii = i < npml ? i : i - nx + w2;
            const int q = (k * ny + j) * w2 + ii;
            const real b = a.bex[ii], aa = a.aex[ii];
            const real p0 = b * a.pex[0][q] + aa * dHz_x;   // Eyx
            const real p1 = b * a.pex[1][q] + aa * dHy_x;   // Ezx
            a.pex[0][q] = p0; a.pex[1][q] = p1;
            ney -= p0;
            nez += p1;
        }
        if (j < npml || j >= ny - npml) {
            const int jj = j < npml ? j : j - ny + w2;
            const int q = (k * w2 + jj) * pitch + i;
            const real b = a.bey[jj], aa = a.aey[jj];
            const real p0 = b * a.pey[0][q] + aa * dHz_y;   // Exy
            const real p1 = b * a.pey[1][q] + aa * dHx_y;   // Ezy
            a.pey[0][q] = p0; a.pey[1][q] = p1;
            nex += p0;
            nez -= p1;
        }
    }
    if (mk & 0x07) {
        const Cpx<real> u = plane_factor(a, k, t.te);
        if (mk & 0x01) nex += src_add(a, 0, col, u);
        if (mk & 0x02) ney += src_add(a, 1, col, u);
        if (mk & 0x04) nez += src_add(a, 2, col, u);
    }
    if (GEN) {
        if (j == 0) { nex = real(0); nez = real(0); }   // PEC: tangential E
        if (i == 0) { ney = real(0); nez = real(0); }
    }
    a.eout[0][g] = nex; a.eout[1][g] = ney; a.eout[2][g] = nez;

    // ---- fluence of step n at the cell centre (i+1/2, j+1/2, k+1/2): E^n over
    // four edges, Hbar over two faces and two times (1/16 folded into dt16)
    if (a.fluence) {
        const real hx_ip = N.template H<0, 1, 0, 0>(hsrc);
        const real hy_jp = N.template H<1, 0, 1, 0>(hsrc);
        const real hz_kp = N.template H<2, 0, 0, 1>(hsrc);
        const real cx = (ex + N.E(0, 0, 1, 0)) + (N.E(0, 0, 0, 1) + N.E(0, 0, 1, 1));
        const real cy = (ey + N.E(1, 1, 0, 0)) + (N.E(1, 0, 0, 1) + N.E(1, 1, 0, 1));
        const real cc = (ez + N.E(2, 1, 0, 0)) + (N.E(2, 0, 1, 0) + N.E(2, 1, 1, 0));
        const real hbx = (N.Ho(0, 0, 0, 0) + hx) + (N.Ho(0, 1, 0, 0) + hx_ip);
        const real hby = (N.Ho(1, 0, 0, 0) + hy) + (N.Ho(1, 0, 1, 0) + hy_jp);
        const real hbz = (N.Ho(2, 0, 0, 0) + hz) + (N.Ho(2, 0, 0, 1) + hz_kp);
        const real sx = cy * hbz - cc * hby;
        const real sy = cc * hbx - cx * hbz;
        const real sz = cx * hby - cy * hbx;
        acc_t* F = static_cast<acc_t*>(a.fluence);
        const real dt16 = real(a.dt16);
        F[g] = Acc::add(F[g], vec_norm(sx * sx + sy * sy + sz * sz) * dt16);
    }
}

// Grid: (ceil(nx/32), ceil(ny/TY), nz) CTAs of 32 x TY threads, one cell each.
template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_step_cell(const StepArgs<real> a, const StepTime<real> t)
{
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY, k = blockIdx.z;
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    const bool gen = i0 == 0 || j0 == 0 || i0 + 32 >= nx || j0 + TY >= ny ||
                     (npml > 0 && (i0 - 1 < npml || i0 + 32 >= nx - npml || j0 - 1 < npml || j0 + TY >= ny - npml));
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (gen) step_cell<real, true>(a, t, i, j, k);
    else step_cell<real, false>(a, t, i, j, k);
}

}  // namespace fdtd
