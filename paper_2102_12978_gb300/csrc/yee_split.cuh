// yee_split.cuh -- the Yee step as two streaming passes over the grid.
//
// Pass 1 (yee_h_pass): H^{n-1/2} -> H^{n+1/2} (curl of E^n, CPML psi of the
// H side, soft source at (n+1/2) dt), Section 4 / Eq. 13.
// Pass 2 (yee_e_pass): E^n -> E^{n+1} (curl of H^{n+1/2}, CPML psi of the E
// side, PEC walls, soft source at (n+1) dt) and, in the same pass, the
// fluence term |E^n_c x Hbar^n_c| dt of every cell (Section 2), with Hbar the
// mean of H^{n-1/2} and H^{n+1/2}.
//
// One thread owns one (i, j) column of a 32 x TY tile and marches a z segment
// [kb, ke), keeping the values its next plane shares with this one in
// registers (E^n and Hz of plane k+1, the +x / +y neighbours the fluence
// needs at k+1, Hx / Hy of plane k-1); the other neighbours come through the
// L1 / L2 caches from the loads of adjacent threads.  There is no halo
// recompute and no shared-memory staging: every cell's H and E are computed
// once, at the price of reading E^n twice and H^{n+1/2} once more than the
// single fused pass (100 instead of 64 bytes per cell outside the CPML).
// Both passes run every thread of a block in one of three specialisations:
// blocks that touch a wall, the last (ragged) tile of an axis or the CPML
// shell compile every check in; interior blocks holding antenna cells add
// only the source; plain interior blocks have neither.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "yee_fused.cuh"
#include "yee_tma.cuh"

namespace fdtd {

template <typename real>
__device__ __forceinline__ real ldro(const real* p)
{
    return __ldg(p);
}

// Class of a split-pass block: gen = it needs the wall / ragged / CPML
// checks, src = (interior) it holds antenna cells.  Block-uniform.
template <typename real, int TY>
__device__ __forceinline__ void split_class(const StepArgs<real>& a, int i0, int j0, bool& gen, bool& src)
{
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    gen = i0 == 0 || j0 == 0 || i0 + 32 >= nx || j0 + TY >= ny ||
          (npml > 0 && (i0 < npml || i0 + 31 >= nx - npml || j0 < npml || j0 + TY - 1 >= ny - npml));
    src = false;
    if (!gen && a.smask) {
        const bool mine = a.smask[(j0 + threadIdx.y) * nx + i0 + threadIdx.x] != 0;
        src = __syncthreads_or(mine) != 0;
    }
}

// Per-plane source factors f e^{i (beta z_k - omega t)} of the planes
// [kb, ke) into u (phase in FP64, stored in the field precision).  t_half:
// 0.5 for the H time (n + 1/2) dt, 1.0 for the E time (n + 1) dt.
template <typename real>
__device__ __forceinline__ void split_factors(const StepArgs<real>& a, long long n, double t_half, int kb, int ke,
                                              Cpx<real>* u, double* tf)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    if (tid == 0) {
        double c, s, f;
        source_time(a.st, (double(n) + t_half) * a.dt, c, s, f);
        tf[0] = c; tf[1] = s; tf[2] = f;
    }
    __syncthreads();
    for (int q = tid; q < ke - kb; q += nt) {
        const double2 z = a.zph[kb + q];
        u[q].x = real((z.x * tf[0] + z.y * tf[1]) * tf[2]);
        u[q].y = real((z.y * tf[0] - z.x * tf[1]) * tf[2]);
    }
    __syncthreads();
}

// H^{n+1/2} of the column (i, j) over planes [kb, ke).
template <typename real, bool GEN, bool SRC>
__device__ __forceinline__ void h_column(const StepArgs<real>& a, const Cpx<real>* __restrict__ u, int i, int j,
                                         int kb, int ke)
{
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    if (GEN && (i >= nx || j >= ny)) return;
    const int plane = pitch * ny, col = j * pitch + i;
    const bool xin = !GEN || i + 1 < nx;   // E at i+1 exists (else the virtual wall: 0)
    const bool yin = !GEN || j + 1 < ny;
    const real chx = a.chx[i], chy = a.chy[j], cz = a.cz;
    const int npml = a.npml, w2 = 2 * npml;
    int ii = -1, jj = -1;
    if (GEN && npml > 0 && (i < npml || i >= nx - npml)) ii = i < npml ? i : i - nx + w2;
    if (GEN && npml > 0 && (j < npml || j >= ny - npml)) jj = j < npml ? j : j - ny + w2;
    real bx = 0, ax = 0, by = 0, ay = 0;
    if (GEN && ii >= 0) { bx = a.bhx[ii]; ax = a.ahx[ii]; }
    if (GEN && jj >= 0) { by = a.bhy[jj]; ay = a.ahy[jj]; }
    uint8_t mk = 0;
    if (SRC && a.smask) mk = a.smask[j * nx + i] & 0x38;
    const int ncol = nx * ny, scol = j * nx + i;
    const Cpx<real>* B = static_cast<const Cpx<real>*>(a.scoefr);
    Cpx<real> b3 = {0, 0}, b4 = {0, 0}, b5 = {0, 0};
    if (SRC && mk) {
        if (mk & 0x08) b3 = B[3 * ncol + scol];
        if (mk & 0x10) b4 = B[4 * ncol + scol];
        if (mk & 0x20) b5 = B[5 * ncol + scol];
    }
    const real* __restrict__ Ex = a.ein[0];
    const real* __restrict__ Ey = a.ein[1];
    const real* __restrict__ Ez = a.ein[2];

    int g = kb * plane + col;
    real ex0 = ldro(Ex + g), ey0 = ldro(Ey + g), ez0 = ldro(Ez + g);
    #pragma unroll 2
    for (int k = kb; k < ke; ++k) {
        const int gn = (k + 1 == nz ? 0 : k + 1) * plane + col;
        const real ex1 = ldro(Ex + gn), ey1 = ldro(Ey + gn), ez1 = ldro(Ez + gn);
        const real ezj = yin ? ldro(Ez + g + pitch) : real(0);
        const real exj = yin ? ldro(Ex + g + pitch) : real(0);
        const real ezi = xin ? ldro(Ez + g + 1) : real(0);
        const real eyi = xin ? ldro(Ey + g + 1) : real(0);
        real hx = ldro(a.hin[0] + g), hy = ldro(a.hin[1] + g), hz = ldro(a.hin[2] + g);
        const real dEz_y = ezj - ez0, dEy_z = ey1 - ey0, dEx_z = ex1 - ex0;
        const real dEz_x = ezi - ez0, dEy_x = eyi - ey0, dEx_y = exj - ex0;
        hx = hx - chy * dEz_y + cz * dEy_z;
        hy = hy - cz * dEx_z + chx * dEz_x;
        hz = hz - chx * dEy_x + chy * dEx_y;
        if (GEN && ii >= 0) {
            const int q = (k * ny + j) * w2 + ii;
            const real p0 = bx * a.phx_in[0][q] + ax * dEz_x;   // Hyx
            const real p1 = bx * a.phx_in[1][q] + ax * dEy_x;   // Hzx
            hy += p0;
            hz -= p1;
            a.phx_out[0][q] = p0; a.phx_out[1][q] = p1;
        }
        if (GEN && jj >= 0) {
            const int q = (k * w2 + jj) * pitch + i;
            const real p0 = by * a.phy_in[0][q] + ay * dEz_y;   // Hxy
            const real p1 = by * a.phy_in[1][q] + ay * dEx_y;   // Hzy
            hx -= p0;
            hz += p1;
            a.phy_out[0][q] = p0; a.phy_out[1][q] = p1;
        }
        if (SRC && mk) {
            const Cpx<real> w = u[k - kb];
            if (mk & 0x08) hx += b3.x * w.x - b3.y * w.y;
            if (mk & 0x10) hy += b4.x * w.x - b4.y * w.y;
            if (mk & 0x20) hz += b5.x * w.x - b5.y * w.y;
        }
        a.hout[0][g] = hx; a.hout[1][g] = hy; a.hout[2][g] = hz;
        ex0 = ex1; ey0 = ey1; ez0 = ez1;
        g += plane;
    }
}

// E^{n+1} and (FLU) the fluence term of the column (i, j) over planes [kb, ke).
template <typename real, bool GEN, bool SRC, bool FLU>
__device__ __forceinline__ void e_column(const StepArgs<real>& a, const Cpx<real>* __restrict__ u, int i, int j,
                                         int kb, int ke)
{
    using Acc = FluAcc<real>;
    using acc_t = typename Acc::T;
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    if (GEN && (i >= nx || j >= ny)) return;
    const int plane = pitch * ny, col = j * pitch + i;
    const bool xin = !GEN || i + 1 < nx, yin = !GEN || j + 1 < ny;
    const bool xlo = !GEN || i > 0, ylo = !GEN || j > 0;
    const real cex = a.cex[i], cey = a.cey[j], cz = a.cz;
    const int npml = a.npml, w2 = 2 * npml;
    int ii = -1, jj = -1;
    if (GEN && npml > 0 && (i < npml || i >= nx - npml)) ii = i < npml ? i : i - nx + w2;
    if (GEN && npml > 0 && (j < npml || j >= ny - npml)) jj = j < npml ? j : j - ny + w2;
    real bx = 0, ax = 0, by = 0, ay = 0;
    if (GEN && ii >= 0) { bx = a.bex[ii]; ax = a.aex[ii]; }
    if (GEN && jj >= 0) { by = a.bey[jj]; ay = a.aey[jj]; }
    uint8_t mk = 0;
    if (SRC && a.smask) mk = a.smask[j * nx + i] & 0x07;
    const int ncol = nx * ny, scol = j * nx + i;
    const Cpx<real>* B = static_cast<const Cpx<real>*>(a.scoefr);
    Cpx<real> b0 = {0, 0}, b1 = {0, 0}, b2 = {0, 0};
    if (SRC && mk) {
        if (mk & 0x01) b0 = B[scol];
        if (mk & 0x02) b1 = B[ncol + scol];
        if (mk & 0x04) b2 = B[2 * ncol + scol];
    }
    const real* __restrict__ Ex = a.ein[0];
    const real* __restrict__ Ey = a.ein[1];
    const real* __restrict__ Ez = a.ein[2];
    const real* __restrict__ Hx = a.hout[0];   // H^{n+1/2}
    const real* __restrict__ Hy = a.hout[1];
    const real* __restrict__ Hz = a.hout[2];
    const real* __restrict__ Ox = a.hin[0];    // H^{n-1/2}
    const real* __restrict__ Oy = a.hin[1];
    const real* __restrict__ Oz = a.hin[2];
    acc_t* __restrict__ F = static_cast<acc_t*>(a.fluence);
    const bool do_flu = FLU && F != nullptr;
    const real dt16 = real(a.dt16);

    int g = kb * plane + col;
    const int gm = (kb == 0 ? nz - 1 : kb - 1) * plane + col;
    real ex0 = ldro(Ex + g), ey0 = ldro(Ey + g), ez0 = ldro(Ez + g);
    real hxm = ldro(Hx + gm), hym = ldro(Hy + gm), hz0 = ldro(Hz + g);
    // the plane-k halves of the fluence's z-pair sums, carried from plane to
    // plane (each is the plane-(k+1) half of the plane before): E_x over the
    // y edges, E_y over the x edges, H_z over the two times
    real cxk = 0, cyk = 0, hzk = 0;
    if (do_flu) {
        const real exj0 = yin ? ldro(Ex + g + pitch) : real(0);
        const real eyi0 = xin ? ldro(Ey + g + 1) : real(0);
        cxk = ex0 + exj0;
        cyk = ey0 + eyi0;
        hzk = ldro(Oz + g) + hz0;
    }
    #pragma unroll 2
    for (int k = kb; k < ke; ++k) {
        const int gn = (k + 1 == nz ? 0 : k + 1) * plane + col;
        const real hx = ldro(Hx + g), hy = ldro(Hy + g), hz = hz0;
        const real hyi = xlo ? ldro(Hy + g - 1) : real(0);
        const real hzi = xlo ? ldro(Hz + g - 1) : real(0);
        const real hxj = ylo ? ldro(Hx + g - pitch) : real(0);
        const real hzj = ylo ? ldro(Hz + g - pitch) : real(0);
        const real dHz_y = hz - hzj, dHy_z = hy - hym, dHx_z = hx - hxm;
        const real dHz_x = hz - hzi, dHy_x = hy - hyi, dHx_y = hx - hxj;
        real nex = ex0 + cey * dHz_y - cz * dHy_z;
        real ney = ey0 + cz * dHx_z - cex * dHz_x;
        real nez = ez0 + cex * dHy_x - cey * dHx_y;
        if (GEN && ii >= 0) {
            const int q = (k * ny + j) * w2 + ii;
            const real p0 = bx * a.pex[0][q] + ax * dHz_x;   // Eyx
            const real p1 = bx * a.pex[1][q] + ax * dHy_x;   // Ezx
            a.pex[0][q] = p0; a.pex[1][q] = p1;
            ney -= p0;
            nez += p1;
        }
        if (GEN && jj >= 0) {
            const int q = (k * w2 + jj) * pitch + i;
            const real p0 = by * a.pey[0][q] + ay * dHz_y;   // Exy
            const real p1 = by * a.pey[1][q] + ay * dHx_y;   // Ezy
            a.pey[0][q] = p0; a.pey[1][q] = p1;
            nex += p0;
            nez -= p1;
        }
        if (SRC && mk) {
            const Cpx<real> w = u[k - kb];
            if (mk & 0x01) nex += b0.x * w.x - b0.y * w.y;
            if (mk & 0x02) ney += b1.x * w.x - b1.y * w.y;
            if (mk & 0x04) nez += b2.x * w.x - b2.y * w.y;
        }
        if (GEN) {
            if (j == 0) { nex = real(0); nez = real(0); }   // PEC: tangential E
            if (i == 0) { ney = real(0); nez = real(0); }
        }
        a.eout[0][g] = nex; a.eout[1][g] = ney; a.eout[2][g] = nez;

        const real ex1 = ldro(Ex + gn), ey1 = ldro(Ey + gn), ez1 = ldro(Ez + gn), hz1 = ldro(Hz + gn);
        if (do_flu) {
            // cell centre (i+1/2, j+1/2, k+1/2): E over four edges, Hbar over
            // two faces and two times (the 1/16 is folded into dt16)
            const real exj1 = yin ? ldro(Ex + gn + pitch) : real(0);
            const real eyi1 = xin ? ldro(Ey + gn + 1) : real(0);
            const real ezj = yin ? ldro(Ez + g + pitch) : real(0);
            const real ezi = xin ? ldro(Ez + g + 1) : real(0);
            const real ezij = (xin && yin) ? ldro(Ez + g + pitch + 1) : real(0);
            const real hxi = xin ? ldro(Hx + g + 1) : real(0);
            const real hyj = yin ? ldro(Hy + g + pitch) : real(0);
            const real ox = ldro(Ox + g), oy = ldro(Oy + g), oz1 = ldro(Oz + gn);
            const real oxi = xin ? ldro(Ox + g + 1) : real(0);
            const real oyj = yin ? ldro(Oy + g + pitch) : real(0);
            const real cxk1 = ex1 + exj1, cyk1 = ey1 + eyi1, hzk1 = oz1 + hz1;
            const real cx = cxk + cxk1;
            const real cy = cyk + cyk1;
            const real cz_ = (ez0 + ezi) + (ezj + ezij);
            const real hbx = (ox + hx) + (oxi + hxi);
            const real hby = (oy + hy) + (oyj + hyj);
            const real hbz = hzk + hzk1;
            const real sx = cy * hbz - cz_ * hby;
            const real sy = cz_ * hbx - cx * hbz;
            const real sz = cx * hby - cy * hbx;
            F[g] = Acc::add(F[g], vec_norm(sx * sx + sy * sy + sz * sz) * dt16);
            cxk = cxk1; cyk = cyk1; hzk = hzk1;
        }
        ex0 = ex1; ey0 = ey1; ez0 = ez1; hz0 = hz1;
        hxm = hx; hym = hy;
        g += plane;
    }
}

// Grid: (ceil(nx/32), ceil(ny/TY), ceil(nz/lz)) CTAs of 32 x TY threads;
// dynamic shared memory lz source factors.  yee_e_pass<.., FLU = false> is
// the E pass after yee_hflu_tma, which has added the fluence term.
template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_h_pass(const StepArgs<real> a, long long n, int lz)
{
    extern __shared__ __align__(16) unsigned char split_raw[];
    Cpx<real>* u = reinterpret_cast<Cpx<real>*>(split_raw);
    __shared__ double tf[3];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY, kb = blockIdx.z * lz, ke = min(kb + lz, a.nz);
    bool gen, src;
    split_class<real, TY>(a, i0, j0, gen, src);
    if ((gen || src) && a.smask) split_factors<real>(a, n, 0.5, kb, ke, u, tf);
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (gen) h_column<real, true, true>(a, u, i, j, kb, ke);
    else if (src) h_column<real, false, true>(a, u, i, j, kb, ke);
    else h_column<real, false, false>(a, u, i, j, kb, ke);
}

template <typename real, int TY, bool FLU>
__global__ void __launch_bounds__(32 * TY)
yee_e_pass(const StepArgs<real> a, long long n, int lz)
{
    extern __shared__ __align__(16) unsigned char split_raw[];
    Cpx<real>* u = reinterpret_cast<Cpx<real>*>(split_raw);
    __shared__ double tf[3];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY, kb = blockIdx.z * lz, ke = min(kb + lz, a.nz);
    bool gen, src;
    split_class<real, TY>(a, i0, j0, gen, src);
    if ((gen || src) && a.smask) split_factors<real>(a, n, 1.0, kb, ke, u, tf);
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (gen) e_column<real, true, true, FLU>(a, u, i, j, kb, ke);
    else if (src) e_column<real, false, true, FLU>(a, u, i, j, kb, ke);
    else e_column<real, false, false, FLU>(a, u, i, j, kb, ke);
}

}  // namespace fdtd
