// yee_cell.cuh -- the Yee step as two cell-parallel passes (sm_103a).
//
// yee_h_cell: H^{n-1/2} -> H^{n+1/2} (curl of E^n, CPML psi of the H side,
// soft source at (n+1/2) dt), Section 4 / Eq. 13.
// yee_e_cell: E^n -> E^{n+1} (curl of H^{n+1/2}, CPML psi of the E side,
// PEC walls, soft source at (n+1) dt) and the fluence term
// |E^n_c x Hbar^n_c| dt of every cell (Section 2), Hbar the mean of
// H^{n-1/2} and H^{n+1/2}.
//
// One thread per cell, a CTA per 32 x TY x 1 block of cells: no loop, no
// barrier, no shared memory and few registers, so that an SM holds enough
// warps -- and enough loads in flight -- to stream HBM at close to its copy
// rate.  The +-1 neighbours of a cell are read through the L1 / L2 caches
// (those of the same plane from adjacent threads, those of planes k +- 1
// from the blocks of the neighbouring plane, which run at about the same
// time).  Blocks that touch a wall, a ragged edge or the CPML shell compile
// every check in; the others none.  The source factor f e^{i (beta z_k -
// omega t)} of a plane is the product of a per-plane table e^{i beta z_k}
// and the per-step factor f e^{-i omega t} evaluated on the host in FP64,
// both in the field precision.
//
// Instantiations: yee_h_cell / yee_e_cell for z-periodic grids; *_w with the
// z walls, their z CPML shell and the Bessel-Gauss wall sheet of Section 2
// compiled in (kept apart, so that the periodic kernels carry none of it);
// *_t / *_wt read the step's time factors from a device table (the batched
// graph).  The cell functions also serve the persistent batch kernel, which
// reads fields on the coherent path (template parameter NC = false).  A
// launch covers at most 65535 planes; taller grids are launched in chunks
// starting at plane a.kbase.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "yee_fused.cuh"
#include "yee_tma.cuh"

namespace fdtd {

// f e^{-i Phi} of the antenna at the H time (n + 1/2) dt and the E time
// (n + 1) dt, and of the wall source at the E time.
template <typename real>
struct StepTime {
    Cpx<real> th, te, tw;
};

// The time factors of step n, evaluated on the host in FP64 and rounded to
// the field precision (every launch path of the cell kernels uses this).
// `wall` is the wall source's envelope, or null.
template <typename real>
inline StepTime<real> step_time(const SrcTime& st, const SrcTime* wall, double dt, long long n)
{
    StepTime<real> t;
    double c, sn, f;
    source_time(st, (double(n) + 0.5) * dt, c, sn, f);
    t.th = Cpx<real>{real(f * c), real(-f * sn)};
    source_time(st, (double(n) + 1.0) * dt, c, sn, f);
    t.te = Cpx<real>{real(f * c), real(-f * sn)};
    t.tw = Cpx<real>{real(0), real(0)};
    if (wall) {
        source_time(*wall, (double(n) + 1.0) * dt, c, sn, f);
        t.tw = Cpx<real>{real(f * c), real(-f * sn)};
    }
    return t;
}

// Block classes of the cell passes: a 32 x TY block needs the checks (GEN)
// if its cells or their +x / +y neighbours (and, for the E pass, -x / -y
// neighbours) reach a wall or a ragged edge, or its cells lie in the shell.
template <typename real, int TY>
__host__ __device__ __forceinline__ bool cell_gen_h(const StepArgs<real>& a, int i0, int j0)
{
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    return i0 + 32 >= nx || j0 + TY >= ny ||
           (npml > 0 && (i0 < npml || i0 + 31 >= nx - npml || j0 < npml || j0 + TY - 1 >= ny - npml));
}
template <typename real, int TY>
__host__ __device__ __forceinline__ bool cell_gen_e(const StepArgs<real>& a, int i0, int j0)
{
    return i0 == 0 || j0 == 0 || cell_gen_h<real, TY>(a, i0, j0);
}

// Planes of a z-walled grid that need the checks: the PEC plane k = 0, the
// last plane (its +z neighbours are the wall) and the z CPML shell.
template <typename real>
__device__ __forceinline__ bool cell_gen_z(const StepArgs<real>& a, int k)
{
    return a.zw && (k == 0 || k + 1 == a.nz || k < a.npz || k >= a.nz - a.npz);
}

// Rounding of the source terms pinned by explicit operations (no contraction
// left to the compiler), so that the term added inside a pass and the one
// added by antenna_add round alike.
__device__ __forceinline__ float mul_rn(float x, float y) { return __fmul_rn(x, y); }
__device__ __forceinline__ double mul_rn(double x, double y) { return __dmul_rn(x, y); }
__device__ __forceinline__ float fma_rn(float x, float y, float z) { return __fmaf_rn(x, y, z); }
__device__ __forceinline__ double fma_rn(double x, double y, double z) { return __fma_rn(x, y, z); }

template <typename real>
__device__ __forceinline__ Cpx<real> plane_factor(const StepArgs<real>& a, int k, Cpx<real> t)
{
    const Cpx<real> z = static_cast<const Cpx<real>*>(a.zphr)[k];
    return Cpx<real>{fma_rn(z.x, t.x, -mul_rn(z.y, t.y)), fma_rn(z.x, t.y, mul_rn(z.y, t.x))};
}

template <typename real>
__device__ __forceinline__ real src_add(const StepArgs<real>& a, int c, int col, Cpx<real> u)
{
    const Cpx<real> b = static_cast<const Cpx<real>*>(a.scoefr)[c * a.nx * a.ny + col];
    return fma_rn(b.x, u.x, -mul_rn(b.y, u.y));
}

// The soft source of Eq. 13 for one side of the antenna, as a pass of its
// own over the antenna's columns only: F_c += Re{coef_c u_k} at every
// antenna point (column cols[q], plane k) of the components c0 .. c0 + 2
// (c0 = 0: E, 3: H) the column's mask holds, u_k = e^{i beta z_k} t.  The
// cell passes then run without the source (smask null).  Used by the FP64
// cell passes: there the FP64 pipe charges a warp instruction whatever the
// number of its active lanes, and the antenna's warps hold about two antenna
// lanes of 32, so the source terms cost an order of magnitude more inside the
// passes than here.  The terms are those the passes add, added last as there
// (the antenna lies outside the CPML shell and off the PEC walls).
template <typename real>
__global__ void __launch_bounds__(256)
antenna_add(const StepArgs<real> a, const int* __restrict__ cols, int ncols, int c0, Cpx<real> t,
            real* __restrict__ f0, real* __restrict__ f1, real* __restrict__ f2)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)ncols * a.nz) return;
    const int q = int(idx % ncols), k = int(idx / ncols);
    const int col = cols[q];
    const int j = col / a.nx, i = col - j * a.nx;
    const uint8_t mk = a.smask[col] >> c0;
    const Cpx<real> u = plane_factor(a, k, t);
    const long long g = (long long)k * a.pitch * a.ny + (long long)j * a.pitch + i;
    if (mk & 1) f0[g] = f0[g] + src_add(a, c0, col, u);
    if (mk & 2) f1[g] = f1[g] + src_add(a, c0 + 1, col, u);
    if (mk & 4) f2[g] = f2[g] + src_add(a, c0 + 2, col, u);
}

// Field loads.  NC: the read-only (non-coherent) path, for kernels in which
// no array they read is written by another block -- every single-step pass;
// the L2 fetches 256 bytes per request, so that a warp's 128-byte row also
// brings in the next block's (the blocks run in x order): 1 % on the E pass.
// A kernel that runs several passes reads values other blocks wrote earlier
// in the same launch and takes the coherent L1 path (ld.global.ca) after its
// grid barrier's acquire fence.
__device__ __forceinline__ float ld_nc_l2_256(const float* p)
{
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_nc_l2_256(const double* p)
{
    double v;
    asm("ld.global.nc.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
// The coherent path with the same fetch hint; volatile with a memory
// clobber, so that no load moves across the grid barrier's fences.
__device__ __forceinline__ float ld_ca_l2_256(const float* p)
{
    float v;
    asm volatile("ld.global.ca.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double ld_ca_l2_256(const double* p)
{
    double v;
    asm volatile("ld.global.ca.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
template <bool NC, typename T>
__device__ __forceinline__ T fld(const T* p)
{
    constexpr bool FP = std::is_same<T, float>::value || std::is_same<T, double>::value;
    if constexpr (NC && FP) return ld_nc_l2_256(p);
    else if constexpr (NC) return __ldg(p);
    else if constexpr (FP) return ld_ca_l2_256(p);
    else return __ldca(p);
}

// WALL: the grid has z walls or a wall sheet (compiled into the *_w kernels
// only, so that z-periodic grids run code without any of it).
template <typename real, bool GEN, bool WALL, bool NC = true>
__device__ __forceinline__ void h_cell(const StepArgs<real>& a, Cpx<real> th, int i, int j, int k)
{
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    if (GEN && (i >= nx || j >= ny)) return;
    const int plane = pitch * ny, g = k * plane + j * pitch + i;
    const int gn = (k + 1 == nz) ? g - k * plane : g + plane;
    const real* __restrict__ Ex = a.ein[0];
    const real* __restrict__ Ey = a.ein[1];
    const real* __restrict__ Ez = a.ein[2];
    const bool xin = !GEN || i + 1 < nx, yin = !GEN || j + 1 < ny;
    const bool ztop = WALL && GEN && a.zw && k + 1 == nz;   // E past the +z wall reads zero
    const real ex = fld<NC>(Ex + g), ey = fld<NC>(Ey + g), ez = fld<NC>(Ez + g);
    const real ex1 = ztop ? real(0) : fld<NC>(Ex + gn), ey1 = ztop ? real(0) : fld<NC>(Ey + gn);
    const real ezj = yin ? fld<NC>(Ez + g + pitch) : real(0);
    const real exj = yin ? fld<NC>(Ex + g + pitch) : real(0);
    const real ezi = xin ? fld<NC>(Ez + g + 1) : real(0);
    const real eyi = xin ? fld<NC>(Ey + g + 1) : real(0);
    real hx = fld<NC>(a.hin[0] + g), hy = fld<NC>(a.hin[1] + g), hz = fld<NC>(a.hin[2] + g);
    const real chx = fld<NC>(a.chx + i), chy = fld<NC>(a.chy + j);
    const real cz = (WALL && GEN && a.zw) ? fld<NC>(a.chz + k) : a.cz;
    const real dEz_y = ezj - ez, dEy_z = ey1 - ey, dEx_z = ex1 - ex;
    const real dEz_x = ezi - ez, dEy_x = eyi - ey, dEx_y = exj - ex;
    hx = hx - chy * dEz_y + cz * dEy_z;
    hy = hy - cz * dEx_z + chx * dEz_x;
    hz = hz - chx * dEy_x + chy * dEx_y;
    if (GEN && a.npml > 0) {
        const int npml = a.npml, w2 = 2 * npml;
        if (i < npml || i >= nx - npml) {
            const int ii = i < npml ? i : i - nx + w2;
            const int q = (k * ny + j) * w2 + ii;
            const real b = a.bhx[ii], aa = a.ahx[ii];
            const real p0 = b * a.phx_in[0][q] + aa * dEz_x;   // Hyx
            const real p1 = b * a.phx_in[1][q] + aa * dEy_x;   // Hzx
            hy += p0;
            hz -= p1;
            a.phx_out[0][q] = p0; a.phx_out[1][q] = p1;
        }
        if (j < npml || j >= ny - npml) {
            const int jj = j < npml ? j : j - ny + w2;
            const int q = (k * w2 + jj) * pitch + i;
            const real b = a.bhy[jj], aa = a.ahy[jj];
            const real p0 = b * a.phy_in[0][q] + aa * dEz_y;   // Hxy
            const real p1 = b * a.phy_in[1][q] + aa * dEx_y;   // Hzy
            hx -= p0;
            hz += p1;
            a.phy_out[0][q] = p0; a.phy_out[1][q] = p1;
        }
    }
    if (WALL && GEN && a.npz > 0 && (k < a.npz || k >= nz - a.npz)) {
        const int w2 = 2 * a.npz, kk = k < a.npz ? k : k - nz + w2;
        const int q = (kk * ny + j) * pitch + i;
        const real b = a.bhz[kk], aa = a.ahz[kk];
        const real p0 = b * a.phz_in[0][q] + aa * dEy_z;   // Hxz
        const real p1 = b * a.phz_in[1][q] + aa * dEx_z;   // Hyz
        hx += p0;
        hy -= p1;
        a.phz_out[0][q] = p0; a.phz_out[1][q] = p1;
    }
    if (a.smask) {
        const int col = j * nx + i;
        const uint8_t mk = fld<NC>(a.smask + col) & 0x38;
        if (mk) {
            const Cpx<real> u = plane_factor(a, k, th);
            if (mk & 0x08) hx += src_add(a, 3, col, u);
            if (mk & 0x10) hy += src_add(a, 4, col, u);
            if (mk & 0x20) hz += src_add(a, 5, col, u);
        }
    }
    a.hout[0][g] = hx; a.hout[1][g] = hy; a.hout[2][g] = hz;
}

// SHY > 0 (FP64 only): the cell's block, of 32 x SHY threads, shares through
// the shared array s_half (3 x 32 x SHY values) the fluence sums that a cell
// and its +y neighbour both form (see the fluence below); every thread of the
// block then runs to the block barrier, a thread past the box on the box's
// last cell of its row / column, storing nothing.
template <typename real, bool GEN, bool WALL, bool NC = true, int SHY = 0>
__device__ __forceinline__ void e_cell(const StepArgs<real>& a, Cpx<real> te, Cpx<real> tw, int i, int j, int k,
                                       real* s_half = nullptr)
{
    using Acc = FluAcc<real>;
    using acc_t = typename Acc::T;
    constexpr bool F64 = std::is_same<real, double>::value;
    static_assert(SHY == 0 || F64, "the shared fluence sums are an FP64 path");
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    const bool live = !GEN || (i < nx && j < ny);   // the cell lies in the box
    if (SHY == 0 && !live) return;
    if (SHY > 0 && GEN) {
        i = i < nx ? i : nx - 1;
        j = j < ny ? j : ny - 1;
    }
    const int plane = pitch * ny, g = k * plane + j * pitch + i;
    const int gm = (k == 0) ? g + (nz - 1) * plane : g - plane;
    const real* __restrict__ Hx = a.hout[0];   // H^{n+1/2}
    const real* __restrict__ Hy = a.hout[1];
    const real* __restrict__ Hz = a.hout[2];
    const bool xlo = !GEN || i > 0, ylo = !GEN || j > 0;
    const bool zbot = WALL && GEN && a.zw && k == 0;   // H below the z = 0 wall reads zero
    const real hx = fld<NC>(Hx + g), hy = fld<NC>(Hy + g), hz = fld<NC>(Hz + g);
    const real hxm = zbot ? real(0) : fld<NC>(Hx + gm), hym = zbot ? real(0) : fld<NC>(Hy + gm);
    const real hyi = xlo ? fld<NC>(Hy + g - 1) : real(0);
    const real hzi = xlo ? fld<NC>(Hz + g - 1) : real(0);
    const real hxj = ylo ? fld<NC>(Hx + g - pitch) : real(0);
    const real hzj = ylo ? fld<NC>(Hz + g - pitch) : real(0);
    const real ex = fld<NC>(a.ein[0] + g), ey = fld<NC>(a.ein[1] + g), ez = fld<NC>(a.ein[2] + g);
    const real cex = fld<NC>(a.cex + i), cey = fld<NC>(a.cey + j);
    const real cz = (WALL && GEN && a.zw) ? fld<NC>(a.cez + k) : a.cz;
    const real dHz_y = hz - hzj, dHy_z = hy - hym, dHx_z = hx - hxm;
    const real dHz_x = hz - hzi, dHy_x = hy - hyi, dHx_y = hx - hxj;
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
            if (live) { a.pex[0][q] = p0; a.pex[1][q] = p1; }
            ney -= p0;
            nez += p1;
        }
        if (j < npml || j >= ny - npml) {
            const int jj = j < npml ? j : j - ny + w2;
            const int q = (k * w2 + jj) * pitch + i;
            const real b = a.bey[jj], aa = a.aey[jj];
            const real p0 = b * a.pey[0][q] + aa * dHz_y;   // Exy
            const real p1 = b * a.pey[1][q] + aa * dHx_y;   // Ezy
            if (live) { a.pey[0][q] = p0; a.pey[1][q] = p1; }
            nex += p0;
            nez -= p1;
        }
    }
    if (WALL && GEN && a.npz > 0 && (k < a.npz || k >= nz - a.npz)) {
        const int w2 = 2 * a.npz, kk = k < a.npz ? k : k - nz + w2;
        const int q = (kk * ny + j) * pitch + i;
        const real b = a.bez[kk], aa = a.aez[kk];
        const real p0 = b * a.pez[0][q] + aa * dHy_z;   // Exz
        const real p1 = b * a.pez[1][q] + aa * dHx_z;   // Eyz
        if (live) { a.pez[0][q] = p0; a.pez[1][q] = p1; }
        nex -= p0;
        ney += p1;
    }
    if (a.smask) {
        const int col = j * nx + i;
        const uint8_t mk = fld<NC>(a.smask + col) & 0x07;
        if (mk) {
            const Cpx<real> u = plane_factor(a, k, te);
            if (mk & 0x01) nex += src_add(a, 0, col, u);
            if (mk & 0x02) ney += src_add(a, 1, col, u);
            if (mk & 0x04) nez += src_add(a, 2, col, u);
        }
    }
    if (WALL && a.wcoefr && k == a.wplane) {   // wall source (Section 2), after the antenna
        const Cpx<real> w = static_cast<const Cpx<real>*>(a.wcoefr)[j * nx + i];
        nex += w.x * tw.x - w.y * tw.y;
    }
    if (GEN) {
        if (j == 0) { nex = real(0); nez = real(0); }   // PEC: tangential E
        if (i == 0) { ney = real(0); nez = real(0); }
        if (zbot) { nex = real(0); ney = real(0); }
    }
    if (live) { a.eout[0][g] = nex; a.eout[1][g] = ney; a.eout[2][g] = nez; }

    if (a.fluence) {
        // cell centre (i+1/2, j+1/2, k+1/2): E over four edges, Hbar over two
        // faces and two times (the 1/16 is folded into dt16)
        const real* __restrict__ Ex = a.ein[0];
        const real* __restrict__ Ey = a.ein[1];
        const real* __restrict__ Ez = a.ein[2];
        const real* __restrict__ Ox = a.hin[0];   // H^{n-1/2}
        const real* __restrict__ Oy = a.hin[1];
        const real* __restrict__ Oz = a.hin[2];
        const int gn = (k + 1 == nz) ? g - k * plane : g + plane;
        const bool xin = !GEN || i + 1 < nx, yin = !GEN || j + 1 < ny;
        const bool zin = !(WALL && GEN && a.zw) || k + 1 < nz;   // plane k+1 inside the z walls
        real cx, cy, cc, hbx, hby, hbz;
        if constexpr (F64) {
            const real ex1 = zin ? fld<NC>(Ex + gn) : real(0), ey1 = zin ? fld<NC>(Ey + gn) : real(0);
            const real eyi = xin ? fld<NC>(Ey + g + 1) : real(0);
            const real eyi1 = (xin && zin) ? fld<NC>(Ey + gn + 1) : real(0);
            const real ezi = xin ? fld<NC>(Ez + g + 1) : real(0);
            const real hxi = xin ? fld<NC>(Hx + g + 1) : real(0);
            const real hz1 = zin ? fld<NC>(Hz + gn) : real(0);
            const real ox = fld<NC>(Ox + g), oy = fld<NC>(Oy + g), oz = fld<NC>(Oz + g);
            const real oz1 = zin ? fld<NC>(Oz + gn) : real(0);
            const real oxi = xin ? fld<NC>(Ox + g + 1) : real(0);
            // The sums over the cell's two y faces (E_x over its four y-z
            // edges, E_z over its four x-y edges, H_y over two faces and two
            // times) are each a row-j half plus a row-(j+1) half, and the
            // row-j half of cell (i, j+1) is the row-(j+1) half of cell
            // (i, j).  SHY blocks take the row-(j+1) halves from the thread of
            // row j+1 where it lies in the block and the box.  E_x's halves
            // are summed over z first on every FP64 path, shared or not, so
            // that all FP64 paths agree bit for bit.
            const real xh = ex + ex1, zh = ez + ezi, yh = oy + hy;   // row j
            real xh1, zh1, yh1;                                       // row j+1
            bool shared = false;
            if constexpr (SHY > 0) {
                constexpr int NB = 32 * SHY;
                const int t = threadIdx.y * 32 + threadIdx.x;
                s_half[t] = xh; s_half[NB + t] = zh; s_half[2 * NB + t] = yh;
                __syncthreads();
                shared = int(threadIdx.y) + 1 < SHY && yin;
                if (shared) { xh1 = s_half[t + 32]; zh1 = s_half[NB + t + 32]; yh1 = s_half[2 * NB + t + 32]; }
            }
            if (!shared) {   // read row j+1 (zero past the box), same operands and order as its thread
                const real e0 = yin ? fld<NC>(Ex + g + pitch) : real(0);
                const real e1 = (yin && zin) ? fld<NC>(Ex + gn + pitch) : real(0);
                const real z0 = yin ? fld<NC>(Ez + g + pitch) : real(0);
                const real z1 = (yin && xin) ? fld<NC>(Ez + g + pitch + 1) : real(0);
                const real o0 = yin ? fld<NC>(Oy + g + pitch) : real(0);
                const real h0 = yin ? fld<NC>(Hy + g + pitch) : real(0);
                xh1 = e0 + e1;
                zh1 = z0 + z1;
                yh1 = o0 + h0;
            }
            cx = xh + xh1;
            cy = (ey + eyi) + (ey1 + eyi1);
            cc = zh + zh1;
            hbx = (ox + hx) + (oxi + hxi);
            hby = yh + yh1;
            hbz = (oz + hz) + (oz1 + hz1);
        } else {
            const real ex1 = zin ? fld<NC>(Ex + gn) : real(0), ey1 = zin ? fld<NC>(Ey + gn) : real(0);
            const real exj = yin ? fld<NC>(Ex + g + pitch) : real(0);
            const real exj1 = (yin && zin) ? fld<NC>(Ex + gn + pitch) : real(0);
            const real eyi = xin ? fld<NC>(Ey + g + 1) : real(0);
            const real eyi1 = (xin && zin) ? fld<NC>(Ey + gn + 1) : real(0);
            const real ezi = xin ? fld<NC>(Ez + g + 1) : real(0);
            const real ezj = yin ? fld<NC>(Ez + g + pitch) : real(0);
            const real ezij = (xin && yin) ? fld<NC>(Ez + g + pitch + 1) : real(0);
            const real hxi = xin ? fld<NC>(Hx + g + 1) : real(0);
            const real hyj = yin ? fld<NC>(Hy + g + pitch) : real(0);
            const real hz1 = zin ? fld<NC>(Hz + gn) : real(0);
            const real ox = fld<NC>(Ox + g), oy = fld<NC>(Oy + g), oz = fld<NC>(Oz + g);
            const real oz1 = zin ? fld<NC>(Oz + gn) : real(0);
            const real oxi = xin ? fld<NC>(Ox + g + 1) : real(0);
            const real oyj = yin ? fld<NC>(Oy + g + pitch) : real(0);
            cx = (ex + exj) + (ex1 + exj1);
            cy = (ey + eyi) + (ey1 + eyi1);
            cc = (ez + ezi) + (ezj + ezij);
            hbx = (ox + hx) + (oxi + hxi);
            hby = (oy + hy) + (oyj + hyj);
            hbz = (oz + hz) + (oz1 + hz1);
        }
        const real sx = cy * hbz - cc * hby;
        const real sy = cc * hbx - cx * hbz;
        const real sz = cx * hby - cy * hbx;
        acc_t* F = static_cast<acc_t*>(a.fluence);
        const real dt16 = real(a.dt16);
        if (live) F[g] = Acc::add(F[g], vec_norm(sx * sx + sy * sy + sz * sz) * dt16);
    }
}

// Grid: (ceil(nx/32), ceil(ny/TY), planes) CTAs of 32 x TY threads, one cell
// each, for planes a.kbase .. a.kbase + gridDim.z - 1 (all planes, or one
// chunk of at most 65535).
// The H pass takes the blocks in launch order, the E pass in reverse order:
// it starts on the planes the H pass touched last, which are still in L2, and
// ends where the next H pass starts.
template <typename real, int TY, bool WALL>
__device__ __forceinline__ void h_block(const StepArgs<real>& a, Cpx<real> th)
{
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY, k = a.kbase + int(blockIdx.z);
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (cell_gen_h<real, TY>(a, i0, j0) || (WALL && cell_gen_z(a, k))) h_cell<real, true, WALL>(a, th, i, j, k);
    else h_cell<real, false, WALL>(a, th, i, j, k);
}

template <typename real, int TY, bool WALL>
__device__ __forceinline__ void e_block(const StepArgs<real>& a, Cpx<real> te, Cpx<real> tw)
{
    const int i0 = (gridDim.x - 1 - blockIdx.x) * 32, j0 = (gridDim.y - 1 - blockIdx.y) * TY;
    const int k = a.kbase + int(gridDim.z - 1 - blockIdx.z);
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    constexpr int SHY = std::is_same<real, double>::value ? TY : 0;   // FP64: fluence sums shared along y
    __shared__ real s_half[SHY > 0 ? 3 * 32 * SHY : 1];
    if (cell_gen_e<real, TY>(a, i0, j0) || (WALL && cell_gen_z(a, k)))
        e_cell<real, true, WALL, true, SHY>(a, te, tw, i, j, k, s_half);
    else e_cell<real, false, WALL, true, SHY>(a, te, tw, i, j, k, s_half);
}

// z-periodic grids without a wall sheet.
template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_h_cell(const StepArgs<real> a, const StepTime<real> t)
{
    h_block<real, TY, false>(a, t.th);
}

template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_e_cell(const StepArgs<real> a, const StepTime<real> t)
{
    e_block<real, TY, false>(a, t.te, t.tw);
}

// Grids with z walls or a wall sheet.  Register budgets: the H pass 32 (2048
// threads per SM), the E pass 40 (FP32, 1536 threads) or 64 (FP64, 1024
// threads), the counts of the kernels above; left to itself the compiler
// spends more on the wall code and loses resident warps.
template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY, 2048 / (32 * TY))
yee_h_cell_w(const StepArgs<real> a, const StepTime<real> t)
{
    h_block<real, TY, true>(a, t.th);
}

template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY, (sizeof(real) == 8 ? 1024 : 1536) / (32 * TY))
yee_e_cell_w(const StepArgs<real> a, const StepTime<real> t)
{
    e_block<real, TY, true>(a, t.te, t.tw);
}

// The same passes with the step's time factors read from a device table
// (times[index]): the batched sweep replays a CUDA graph whose steps take
// their source phase from a table refreshed before each replay.
template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_h_cell_t(const StepArgs<real> a, const StepTime<real>* __restrict__ times, int index)
{
    h_block<real, TY, false>(a, times[index].th);
}

template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_e_cell_t(const StepArgs<real> a, const StepTime<real>* __restrict__ times, int index)
{
    e_block<real, TY, false>(a, times[index].te, Cpx<real>{real(0), real(0)});
}

template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY, 2048 / (32 * TY))
yee_h_cell_wt(const StepArgs<real> a, const StepTime<real>* __restrict__ times, int index)
{
    h_block<real, TY, true>(a, times[index].th);
}

template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY, (sizeof(real) == 8 ? 1024 : 1536) / (32 * TY))
yee_e_cell_wt(const StepArgs<real> a, const StepTime<real>* __restrict__ times, int index)
{
    e_block<real, TY, true>(a, times[index].te, times[index].tw);
}

}  // namespace fdtd
