// yee_tma.cuh -- the fused Yee step with TMA-staged planes (sm_103a).
//
// Same arithmetic and work decomposition as yee_step_fused (one CTA per
// 32 x TY column tile and z segment, H recomputed on a one-cell low halo, E
// update and fluence in the same pass, Section 4 / Eq. 13 / Section 2), but
// the inputs of each z plane are moved by the Tensor Memory Accelerator:
//   * one thread issues cp.async.bulk.tensor.3d box loads of E^n (tile plus a
//     one-cell halo on every side), H^{n-1/2} (tile plus the low halo) and the
//     old fluence of the plane into an S-stage shared-memory ring, S-2 planes
//     ahead of use; each stage completes on its own mbarrier (expect_tx);
//   * out-of-range box elements (i < 0, i >= nx, j < 0, j >= ny) are filled
//     with zeros by the TMA unit, which is exactly the PEC wall value the
//     stencil needs there;
//   * x box starts are rounded down to a 16-byte boundary (i0 - 4 for FP32,
//     i0 - 2 for FP64) so every copy starts aligned.
// Every wait is bounded (about two seconds of SM clock); on expiry the CTA
// raises the grid's error word, stops marching, drains its own copies and
// returns, so the host sees FDTD_ETIMEOUT instead of a hung device.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "yee_fused.cuh"

namespace fdtd {

struct TmaMaps {
    CUtensorMap e[3];   // E^n of the copy being read
    CUtensorMap h[3];   // H^{n-1/2} of the copy being read
    CUtensorMap f;      // fluence accumulator (8 bytes per cell)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: about 2^32 SM cycles (~2 s at 2 GHz) before giving up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 32)) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Box and ring geometry of a tile of 32 x TR columns (TR rows).
template <typename real, int TR>
struct TmaTile {
    static constexpr int TX = 32;
    static constexpr int XA = 16 / int(sizeof(real));   // x alignment in elements
    static constexpr int BX = TX + 2 * XA;              // E / H box width
    static constexpr int EBY = TR + 2;                  // E box rows (j0-1 .. j0+TR)
    static constexpr int HBY = TR + 2;                  // H box rows (j0-1 .. j0+TR; the last row
                                                        // is read only at the +y wall, as zeros)
    static constexpr int FBX = TX + 2, FBY = TR + 1;    // fluence box (i0-2 .., j0-1 ..)
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t EB = al(size_t(BX) * EBY * sizeof(real));
    static constexpr size_t HB = al(size_t(BX) * HBY * sizeof(real));
    static constexpr size_t FB = al(size_t(FBX) * FBY * 8);
    static constexpr size_t STAGE = 3 * EB + 3 * HB + FB;
    static constexpr int PX = TX + 2, PY = TR + 2, P = PX * PY;   // H^{n+1/2} ring
    static constexpr uint32_t E_BYTES = uint32_t(BX * EBY * sizeof(real));
    static constexpr uint32_t H_BYTES = uint32_t(BX * HBY * sizeof(real));
    static constexpr uint32_t F_BYTES = uint32_t(FBX * FBY * 8);
    // stages + 3-slot ring of H^{n+1/2} + per-plane source factors (E and H
    // times, lz + 3 planes) + mbarriers + alignment slack
    static constexpr size_t smem_bytes(int S, int lz)
    {
        return S * STAGE + 9 * size_t(P) * sizeof(real) + 2 * size_t(lz + 3) * 2 * sizeof(real) + S * 8 + 128;
    }
};

template <typename real> struct Cpx { real x, y; };

// |S| from |S|^2.
//
// FP64: one Newton step on s^2 = x (Heron's method, s <- (s + x / s) / 2,
// written with r ~ 1/sqrt(x) as s1 = s0 + (x - s0^2) r / 2 with s0 = x r),
// seeded by the single-precision reciprocal square root.  The seed's float
// argument and the conversion of r back to FP64 are made from the double's
// bits with integer operations (x rounded toward zero to 24 bits; r exact),
// and r / 2 by lowering r's exponent, so the FP64 pipe -- 1/64 of the FP32
// rate on this GPU -- runs three operations (a multiply and two fused
// multiply-adds).  With the seed's relative error e (rsqrtf's two ulp plus the
// truncation of x: |e| < 2^-21.4), the step leaves -3 e^2 / 2 (< 2^-42, 2.3e-13)
// plus the FP64 rounding of the three operations.  x = 0 returns 0; x outside
// float's normal range [2^-126, 2^128) (or not finite) takes sqrt().
//
// FP32: x * rsqrt(x) (a few ulp, far inside the FP32 tolerance of the
// fluence), which avoids the long correctly-rounded sequence per cell.
__device__ __forceinline__ double vec_norm(double x)
{
    const int hi = __double2hiint(x);
    const unsigned lo = static_cast<unsigned>(__double2loint(x));
    const int e = (hi >> 20) & 0x7ff;   // biased exponent (x >= 0)
    if (e >= 1023 - 126 && e <= 1023 + 127) {
        // float of x: exponent rebiased by 1023 - 127, the top 23 of 52 mantissa bits
        const unsigned fb = (static_cast<unsigned>(e - 896) << 23) | ((static_cast<unsigned>(hi) & 0xfffffu) << 3) |
                            (lo >> 29);
        const unsigned rb = __float_as_uint(rsqrtf(__uint_as_float(fb)));   // in (2^-64, 2^63]
        // the double of r: exponent rebiased by 896, the 23 mantissa bits on top
        const int rhi = static_cast<int>((((rb >> 23) + 896u) << 20) | ((rb & 0x7fffffu) >> 3));
        const int rlo = static_cast<int>(rb << 29);
        const double r = __hiloint2double(rhi, rlo);
        const double h = __hiloint2double(rhi - (1 << 20), rlo);   // r / 2
        const double s0 = x * r;
        return fma(fma(-s0, s0, x), h, s0);
    }
    if ((hi | static_cast<int>(lo)) == 0) return 0.0;
    return sqrt(x);
}
__device__ __forceinline__ float vec_norm(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// Per-column constants of one H cell: curl coefficients, CPML shell indices
// (-1 outside the shell; the profile values are re-read from the small,
// cache-resident tables), antenna mask.
template <typename real>
struct HCol {
    bool valid;
    int ci, cj;
    real chx, chy;
    int ii, jj;            // x / y shell index, or -1
    uint8_t mk;
};

template <typename real, bool GEN, bool SRC>
__device__ __forceinline__ HCol<real> make_hcol(const StepArgs<real>& a, int ci, int cj, bool valid)
{
    HCol<real> c;
    c.valid = valid;
    c.ci = ci; c.cj = cj;
    c.chx = real(0); c.chy = real(0); c.ii = -1; c.jj = -1; c.mk = 0;
    if (!valid) return c;
    c.chx = a.chx[ci]; c.chy = a.chy[cj];
    const int npml = a.npml, w2 = 2 * npml;
    if (GEN && npml > 0 && (ci < npml || ci >= a.nx - npml)) c.ii = ci < npml ? ci : ci - a.nx + w2;
    if (GEN && npml > 0 && (cj < npml || cj >= a.ny - npml)) c.jj = cj < npml ? cj : cj - a.ny + w2;
    if (SRC && a.smask) c.mk = a.smask[cj * a.nx + ci];
    return c;
}

// H^{n+1/2} of one cell from the staged E planes k (e0*) and k+1 (e1*); the
// CPML psi of the H side (old values in pp, prefetched from the read copy)
// is written, if `store`, to the write copy.
template <typename real, int BX, bool GEN, bool SRC>
__device__ __forceinline__ void tma_compute_h(const StepArgs<real>& a, const HCol<real>& c,
                                              const real* __restrict__ e0x, const real* __restrict__ e0y,
                                              const real* __restrict__ e0z, const real* __restrict__ e1x,
                                              const real* __restrict__ e1y, int idx, int kw, real& hx, real& hy,
                                              real& hz, Cpx<real> u, bool store, const real (&pp)[4])
{
    const real ex = e0x[idx], ey = e0y[idx], ez = e0z[idx];
    const real dEz_y = e0z[idx + BX] - ez;
    const real dEy_z = e1y[idx] - ey;
    const real dEx_z = e1x[idx] - ex;
    const real dEz_x = e0z[idx + 1] - ez;
    const real dEy_x = e0y[idx + 1] - ey;
    const real dEx_y = e0x[idx + BX] - ex;
    hx = hx - c.chy * dEz_y + a.cz * dEy_z;
    hy = hy - a.cz * dEx_z + c.chx * dEz_x;
    hz = hz - c.chx * dEy_x + c.chy * dEx_y;
    if (GEN && c.ii >= 0) {
        const int w2 = 2 * a.npml;
        const int q = (kw * a.ny + c.cj) * w2 + c.ii;
        const real b = a.bhx[c.ii], aa = a.ahx[c.ii];
        const real p0 = b * pp[0] + aa * dEz_x;   // Hyx (old value prefetched)
        const real p1 = b * pp[1] + aa * dEy_x;   // Hzx
        hy += p0;
        hz -= p1;
        if (store) { a.phx_out[0][q] = p0; a.phx_out[1][q] = p1; }
    }
    if (GEN && c.jj >= 0) {
        const int w2 = 2 * a.npml;
        const int q = (kw * w2 + c.jj) * a.pitch + c.ci;
        const real b = a.bhy[c.jj], aa = a.ahy[c.jj];
        const real p0 = b * pp[2] + aa * dEz_y;   // Hxy
        const real p1 = b * pp[3] + aa * dEx_y;   // Hzy
        hx -= p0;
        hz += p1;
        if (store) { a.phy_out[0][q] = p0; a.phy_out[1][q] = p1; }
    }
    if (SRC && (c.mk & 0x38)) {
        // soft source: Re{ B u }, u = f e^{i (beta z_k - Phi)} of this plane
        const int ncol = a.nx * a.ny, col = c.cj * a.nx + c.ci;
        const Cpx<real>* B = static_cast<const Cpx<real>*>(a.scoefr);
        if (c.mk & 0x08) { const Cpx<real> b = B[3 * ncol + col]; hx += b.x * u.x - b.y * u.y; }
        if (c.mk & 0x10) { const Cpx<real> b = B[4 * ncol + col]; hy += b.x * u.x - b.y * u.y; }
        if (c.mk & 0x20) { const Cpx<real> b = B[5 * ncol + col]; hz += b.x * u.x - b.y * u.y; }
    }
}

// Fluence term of one cell: |E_c x Hbar_c| dt added to the accumulator.
// em*/ek*: staged E planes of the cell (k) and of k+1 (box index ce);
// hm/hk: staged H^{n-1/2} boxes of planes k, k+1 (box index ce, component
// stride HS); sm/sk: H^{n+1/2} ring slots of planes k, k+1 (ring index cs).
// The means' factors (1/4 for E, 1/4 for H-bar) are folded into dt16.
template <typename real, int BX, int PX, int P, int HS>
__device__ __forceinline__ void tma_fluence_cell(const real* __restrict__ emx, const real* __restrict__ emy,
                                                 const real* __restrict__ emz, const real* __restrict__ ekx,
                                                 const real* __restrict__ eky, const real* __restrict__ hm,
                                                 const real* __restrict__ hk, const real* __restrict__ sm,
                                                 const real* __restrict__ sk, int ce, int cs,
                                                 const typename FluAcc<real>::T& fo, real dt16,
                                                 typename FluAcc<real>::T* F, int g)
{
    const real ex = (emx[ce] + emx[ce + BX]) + (ekx[ce] + ekx[ce + BX]);
    const real ey = (emy[ce] + emy[ce + 1]) + (eky[ce] + eky[ce + 1]);
    const real ez = (emz[ce] + emz[ce + 1]) + (emz[ce + BX] + emz[ce + BX + 1]);
    const real hx = (hm[ce] + sm[cs]) + (hm[ce + 1] + sm[cs + 1]);
    const real hy = (hm[HS + ce] + sm[P + cs]) + (hm[HS + ce + BX] + sm[P + cs + PX]);
    const real hz = (hm[2 * HS + ce] + sm[2 * P + cs]) + (hk[2 * HS + ce] + sk[2 * P + cs]);
    const real sx = ey * hz - ez * hy;
    const real sy = ez * hx - ex * hz;
    const real sz = ex * hy - ey * hx;
    F[g] = FluAcc<real>::add(fo, vec_norm(sx * sx + sy * sy + sz * sz) * dt16);
}

// Shared memory of one CTA running tma_march.
template <typename real, int TR, int S>
struct MarchSmem {
    unsigned char* base;   // S stages
    real* sH;              // [3][3][P] ring of H^{n+1/2}
    Cpx<real>* uE;         // per-plane source factor at the E time, lz + 3 planes
    Cpx<real>* uH;         // the same at the H time
    uint64_t* bars;        // S mbarriers
    double* tf;            // 6 time factors
    int* abort_flag;
};

// One CTA of TW = TR / R warps marches one (32 x TR) x [kb, ke) block of a
// grid through one Yee step; each thread owns R rows of its column (rows
// ty, ty + TW, ...), which shares the per-plane control, waits and barrier
// between R independent cells.  gq0 is the CTA's running plane counter
// (stage = gq % S, mbarrier parity = (gq / S) & 1), so that a persistent CTA
// can march many blocks with its mbarriers initialised once.  Returns the
// updated counter, or -1 after a timed-out wait (the error word is raised).
// GEN: the block may touch the CPML shell, a PEC wall or the last (wall or
// ragged) tile of an axis, and every per-cell check is compiled in; !GEN
// compiles them out.  SRC: the block holds antenna cells.
template <typename real, int TR, int R, int S, bool GEN, bool SRC>
__device__ __forceinline__ int tma_march(const StepArgs<real>& a, const TmaMaps& m, long long n, int i0, int j0,
                                         int kb, int ke, int* err, const MarchSmem<real, TR, S>& sm, int gq0)
{
    static_assert(S >= 5, "the ring needs S >= 5 stages (lead of S-3 planes)");
    static_assert(TR % R == 0, "tile rows must be a multiple of the rows per thread");
    using T = TmaTile<real, TR>;
    using Acc = FluAcc<real>;
    using acc_t = typename Acc::T;
    constexpr int TX = T::TX, BX = T::BX, XA = T::XA, PX = T::PX, P = T::P, FBX = T::FBX;
    constexpr int TW = TR / R;                       // warps
    constexpr int NT = 32 * TW;
    constexpr int HS = int(T::HB / sizeof(real));
    static_assert(TR + 1 <= 32, "the halo column must fit one warp");
    static_assert(TW >= 2, "the halo row and column need two warps");
    unsigned char* base = sm.base;
    real* sH = sm.sH;
    uint64_t* bars = sm.bars;
    double* tf = sm.tf;
    int& abort_flag = *sm.abort_flag;

    const int tx = threadIdx.x, tw = threadIdx.y, tid = tw * TX + tx;
    constexpr int PRODUCER = (TW - 1) * 32;          // lane 0 of the last warp issues TMA
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    const int plane = pitch * ny;
    const int w2 = 2 * a.npml, psx_plane = ny * w2, psy_plane = w2 * pitch;
    const int i = i0 + tx;
    const bool do_flu = a.fluence != nullptr;
    acc_t* F = static_cast<acc_t*>(a.fluence);
    const real dtr = real(a.dt);
    const int Q = ke - kb + 3;                       // E planes kb-1 .. ke+1

    auto stage = [&](int s) { return base + s * T::STAGE; };

    // ---- TMA producer: plane q of this block into stage (gq0 + q) % S
    // test hook: the first CTA arms plane 1's mbarrier but withholds its
    // copies, so that its bounded wait expires (the drain skips that plane)
    const int withheld = (a.fault == 1 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) ? 1 : -1;
    auto issue = [&](int q) {
        const int p = kb - 1 + q;
        const int pw = p < 0 ? p + nz : (p >= nz ? p - nz : p);
        const bool needH = p <= ke;
        const bool needF = do_flu && p >= kb && p <= ke - 1;
        const int s = (gq0 + q) % S;
        uint64_t* bar = &bars[s];
        unsigned char* st = stage(s);
        mbar_expect_tx(bar, 3 * T::E_BYTES + (needH ? 3 * T::H_BYTES : 0u) + (needF ? T::F_BYTES : 0u));
        if (q == withheld) return;
        #pragma unroll
        for (int c = 0; c < 3; ++c) tma_load_3d(st + c * T::EB, &m.e[c], bar, i0 - XA, j0 - 1, pw);
        if (needH) {
            #pragma unroll
            for (int c = 0; c < 3; ++c) tma_load_3d(st + 3 * T::EB + c * T::HB, &m.h[c], bar, i0 - XA, j0 - 1, pw);
        }
        if (needF) tma_load_3d(st + 3 * T::EB + 3 * T::HB, &m.f, bar, i0 - 2, j0 - 1, pw);
    };

    int issued = 0;
    __syncthreads();   // the previous block's readers of every stage are done
    if (tid == PRODUCER) fence_proxy_async();
    if (tid == 0) {
        double c, s, f;
        source_time(a.st, (double(n) + 0.5) * a.dt, c, s, f);
        tf[3] = c; tf[4] = s; tf[5] = f;
        source_time(a.st, (double(n) + 1.0) * a.dt, c, s, f);
        tf[0] = c; tf[1] = s; tf[2] = f;
    }
    for (int q = tid; q < 9 * P; q += NT) sH[q] = real(0);    // H^{n+1/2} ring
    __syncthreads();
    if (tid == PRODUCER) {
        #pragma unroll 1
        for (; issued < S - 3 && issued < Q; ++issued) issue(issued);
    }
    // source factors f e^{i (beta z_k - omega t')} of every plane of this
    // block, phase in FP64, stored in the field precision
    if (SRC && a.smask) {
        for (int q = tid; q < Q; q += NT) {
            const int p = kb - 1 + q;
            const int pw = p < 0 ? p + nz : (p >= nz ? p - nz : p);
            const double2 z = a.zph[pw];
            sm.uE[q].x = real((z.x * tf[0] + z.y * tf[1]) * tf[2]);
            sm.uE[q].y = real((z.y * tf[0] - z.x * tf[1]) * tf[2]);
            sm.uH[q].x = real((z.x * tf[3] + z.y * tf[4]) * tf[5]);
            sm.uH[q].y = real((z.y * tf[3] - z.x * tf[4]) * tf[5]);
        }
    }

    // ---- per-row constants of this thread's R cells
    int jr[R], so[R], eo[R], gcol[R];
    bool own[R], flu_base[R], xw[R], yw[R];
    HCol<real> co[R];
    real cex = real(0), cey[R];
    int eii[R], ejj[R];                              // E-side CPML shell indices or -1
    #pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ty = tw + r * TW;
        const int j = j0 + ty;
        jr[r] = j;
        so[r] = (ty + 1) * PX + (tx + 1);
        eo[r] = (ty + 1) * BX + (tx + XA);
        gcol[r] = j * pitch + i;
        own[r] = !GEN || ((i < nx) && (j < ny));
        co[r] = make_hcol<real, GEN, SRC>(a, i, j, own[r]);
        cey[r] = own[r] ? a.cey[j] : real(0);
        eii[r] = -1; ejj[r] = -1;
        if (GEN && own[r] && w2 > 0) {
            if (i < a.npml || i >= nx - a.npml) eii[r] = i < a.npml ? i : i - nx + w2;
            if (j < a.npml || j >= ny - a.npml) ejj[r] = j < a.npml ? j : j - ny + w2;
        }
        flu_base[r] = !GEN || ((i >= 1) && (j >= 1) && (i <= nx) && (j <= ny));
        xw[r] = GEN && (tx == TX - 1) && (i == nx - 1) && (j >= 1) && (j <= ny);
        yw[r] = GEN && (ty == TR - 1) && (j == ny - 1) && (i >= 1) && (i <= nx);
    }
    if (own[0]) cex = a.cex[i];
    // halo H cells: the row j0-1 on warp 0, the column i0-1 (TR+1 cells) on
    // warp TW/2, so that no warp carries both
    int hs_h = 0, he_h = 0, hi_h = -1, hj_h = -1;
    if (tw == 0) { hi_h = i0 + tx; hj_h = j0 - 1; hs_h = tx + 1; he_h = tx + XA; }
    else if (tw == TW / 2 && tx <= TR) {
        hi_h = i0 - 1; hj_h = j0 - 1 + tx; hs_h = tx * PX; he_h = tx * BX + XA - 1;
    }
    const bool hvalid = GEN ? (hi_h >= 0 && hi_h < nx && hj_h >= 0 && hj_h < ny) : (hi_h != -1 || hj_h != -1);
    const HCol<real> ch = make_hcol<real, GEN, SRC>(a, hi_h, hj_h, hvalid);

    // CPML psi of the next plane, prefetched into registers one iteration
    // ahead (H side: own and halo cells, read copy; E side: own cells,
    // updated in place)
    real ppo[R][4], ppe[R][4], pph[4] = {0, 0, 0, 0};
    #pragma unroll
    for (int r = 0; r < R; ++r)
        #pragma unroll
        for (int c = 0; c < 4; ++c) { ppo[r][c] = real(0); ppe[r][c] = real(0); }
    auto fetch_psi_h = [&](const HCol<real>& c, int pw, real (&pp)[4]) {
        if (!GEN) return;
        if (c.ii >= 0) {
            const int q = pw * psx_plane + c.cj * w2 + c.ii;
            pp[0] = a.phx_in[0][q]; pp[1] = a.phx_in[1][q];
        }
        if (c.jj >= 0) {
            const int q = pw * psy_plane + c.jj * pitch + c.ci;
            pp[2] = a.phy_in[0][q]; pp[3] = a.phy_in[1][q];
        }
    };
    auto fetch_psi = [&](int pw_h, int pw_e, bool e) {
        if (GEN) {
            #pragma unroll
            for (int r = 0; r < R; ++r) {
                fetch_psi_h(co[r], pw_h, ppo[r]);
                if (e && eii[r] >= 0) {
                    const int q = pw_e * psx_plane + jr[r] * w2 + eii[r];
                    ppe[r][0] = a.pex[0][q]; ppe[r][1] = a.pex[1][q];
                }
                if (e && ejj[r] >= 0) {
                    const int q = pw_e * psy_plane + ejj[r] * pitch + i;
                    ppe[r][2] = a.pey[0][q]; ppe[r][3] = a.pey[1][q];
                }
            }
            fetch_psi_h(ch, pw_h, pph);
        }
    };
    fetch_psi(kb - 1 < 0 ? kb - 1 + nz : kb - 1, 0, false);

    int waited = -1;
    int kw = kb - 1 < 0 ? kb - 1 + nz : kb - 1;    // wrapped plane of iteration k
    int s0 = gq0 % S;                                // stage of plane q
    uint32_t par = uint32_t((gq0 / S) & 1);          // mbarrier parity of plane q
    int r0 = 0, r1 = 2, r2 = 1;                      // H-ring slots of q, q-1, q-2
    #pragma unroll 1
    for (int q = 0; q <= Q - 1; ++q) {
        const int k = kb - 1 + q;
        // wait for plane q+1 (and plane 0 on the first pass)
        bool ok = true;
        if (q == 0) ok = mbar_wait_bounded(&bars[s0], par);
        const int s1 = (s0 + 1 == S) ? 0 : s0 + 1;
        const uint32_t par1 = (s0 + 1 == S) ? (par ^ 1u) : par;
        if (q + 1 <= Q - 1) ok = ok && mbar_wait_bounded(&bars[s1], par1);
        if (ok) waited = q + 1;
        else { abort_flag = 1; atomicOr(err, 1); }
        __syncthreads();   // planes q, q+1 landed; every reader of plane q-3 is done
        if (abort_flag) break;
        if (tid == PRODUCER && issued < Q) { fence_proxy_async(); issue(issued); ++issued; }

        const unsigned char* st0 = stage(s0);
        const real* e0x = reinterpret_cast<const real*>(st0);
        const real* e0y = reinterpret_cast<const real*>(st0 + T::EB);
        const real* e0z = reinterpret_cast<const real*>(st0 + 2 * T::EB);

        // ---- H^{n+1/2} of plane k (tile + low halo)
        if (k <= ke) {
            const unsigned char* stn = stage(s1);
            const real* e1x = reinterpret_cast<const real*>(stn);
            const real* e1y = reinterpret_cast<const real*>(stn + T::EB);
            const real* hb = reinterpret_cast<const real*>(st0 + 3 * T::EB);
            real* hs = sH + r0 * 3 * P;
            const bool write_k = (k >= kb) && (k < ke);
            Cpx<real> uh;
            if (SRC) uh = sm.uH[q];
            #pragma unroll
            for (int r = 0; r < R; ++r) {
                if (co[r].valid) {
                    real hx = hb[eo[r]], hy = hb[HS + eo[r]], hz = hb[2 * HS + eo[r]];
                    tma_compute_h<real, BX, GEN, SRC>(a, co[r], e0x, e0y, e0z, e1x, e1y, eo[r], kw, hx, hy, hz, uh,
                                                      write_k, ppo[r]);
                    hs[so[r]] = hx; hs[P + so[r]] = hy; hs[2 * P + so[r]] = hz;
                    if (write_k) {
                        const int g = kw * plane + gcol[r];
                        a.hout[0][g] = hx; a.hout[1][g] = hy; a.hout[2][g] = hz;
                    }
                }
            }
            if (ch.valid) {
                real hx = hb[he_h], hy = hb[HS + he_h], hz = hb[2 * HS + he_h];
                tma_compute_h<real, BX, GEN, SRC>(a, ch, e0x, e0y, e0z, e1x, e1y, he_h, kw, hx, hy, hz, uh, false,
                                                  pph);
                hs[hs_h] = hx; hs[P + hs_h] = hy; hs[2 * P + hs_h] = hz;
            }
        }

        // ---- E^{n+1} of plane k-1 (needs H^{n+1/2} of planes k-1, k-2)
        const int km = k - 1;
        const int kmw = kw == 0 ? nz - 1 : kw - 1;
        const int sm1 = s0 == 0 ? S - 1 : s0 - 1;
        if (km >= kb && km < ke) {
            const real* h0 = sH + r1 * 3 * P;
            const real* h1 = sH + r2 * 3 * P;
            const unsigned char* stm = stage(sm1);
            const real* epx = reinterpret_cast<const real*>(stm);
            const real* epy = reinterpret_cast<const real*>(stm + T::EB);
            const real* epz = reinterpret_cast<const real*>(stm + 2 * T::EB);
            Cpx<real> ue;
            if (SRC) ue = sm.uE[q - 1];
            #pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!own[r]) continue;
                const int o = so[r];
                const real ex = epx[eo[r]], ey = epy[eo[r]], ez = epz[eo[r]];
                const real hx0 = h0[o], hy0 = h0[P + o], hz0 = h0[2 * P + o];
                const real dHz_y = hz0 - h0[2 * P + o - PX];
                const real dHy_z = hy0 - h1[P + o];
                const real dHx_z = hx0 - h1[o];
                const real dHz_x = hz0 - h0[2 * P + o - 1];
                const real dHy_x = hy0 - h0[P + o - 1];
                const real dHx_y = hx0 - h0[o - PX];
                real nex = ex + cey[r] * dHz_y - a.cz * dHy_z;
                real ney = ey + a.cz * dHx_z - cex * dHz_x;
                real nez = ez + cex * dHy_x - cey[r] * dHx_y;
                if (GEN && eii[r] >= 0) {
                    const int qq = (kmw * ny + jr[r]) * w2 + eii[r];
                    const real b = a.bex[eii[r]], aa = a.aex[eii[r]];
                    const real p0 = b * ppe[r][0] + aa * dHz_x;   // Eyx (old value prefetched)
                    const real p1 = b * ppe[r][1] + aa * dHy_x;   // Ezx
                    a.pex[0][qq] = p0; a.pex[1][qq] = p1;
                    ney -= p0;
                    nez += p1;
                }
                if (GEN && ejj[r] >= 0) {
                    const int qq = (kmw * w2 + ejj[r]) * pitch + i;
                    const real b = a.bey[ejj[r]], aa = a.aey[ejj[r]];
                    const real p0 = b * ppe[r][2] + aa * dHz_y;   // Exy
                    const real p1 = b * ppe[r][3] + aa * dHx_y;   // Ezy
                    a.pey[0][qq] = p0; a.pey[1][qq] = p1;
                    nex += p0;
                    nez -= p1;
                }
                if (SRC && (co[r].mk & 0x07)) {
                    const int ncol = nx * ny, col = jr[r] * nx + i;
                    const Cpx<real>* B = static_cast<const Cpx<real>*>(a.scoefr);
                    if (co[r].mk & 0x01) { const Cpx<real> b = B[col]; nex += b.x * ue.x - b.y * ue.y; }
                    if (co[r].mk & 0x02) { const Cpx<real> b = B[ncol + col]; ney += b.x * ue.x - b.y * ue.y; }
                    if (co[r].mk & 0x04) { const Cpx<real> b = B[2 * ncol + col]; nez += b.x * ue.x - b.y * ue.y; }
                }
                if (GEN) {
                    if (jr[r] == 0) { nex = real(0); nez = real(0); }    // PEC: tangential E
                    if (i == 0) { ney = real(0); nez = real(0); }
                }
                const int g = kmw * plane + gcol[r];
                a.eout[0][g] = nex; a.eout[1][g] = ney; a.eout[2][g] = nez;
            }
        }

        // ---- fluence of plane k-2: E planes k-2, k-1 and H-bar of k-2, k-1
        const int kf = k - 2;
        if (do_flu && kf >= kb && kf < ke) {
            const int kfw = kmw == 0 ? nz - 1 : kmw - 1;
            const int sm2 = sm1 == 0 ? S - 1 : sm1 - 1;
            const unsigned char* sa = stage(sm2);
            const unsigned char* sb = stage(sm1);
            const real* emx = reinterpret_cast<const real*>(sa);
            const real* emy = reinterpret_cast<const real*>(sa + T::EB);
            const real* emz = reinterpret_cast<const real*>(sa + 2 * T::EB);
            const real* ekx = reinterpret_cast<const real*>(sb);
            const real* eky = reinterpret_cast<const real*>(sb + T::EB);
            const acc_t* fo = reinterpret_cast<const acc_t*>(sa + 3 * T::EB + 3 * T::HB);
            const real* hm = reinterpret_cast<const real*>(sa + 3 * T::EB);
            const real* hk = reinterpret_cast<const real*>(sb + 3 * T::EB);
            const real* smm = sH + r2 * 3 * P;
            const real* skk = sH + r1 * 3 * P;
            const real dt16 = dtr * real(0.0625);
            const int gp = kfw * plane;
            #pragma unroll
            for (int r = 0; r < R; ++r) {
                const int ty = tw + r * TW;
                if (flu_base[r])
                    tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, smm, skk, eo[r] - BX - 1,
                                                          so[r] - PX - 1, fo[ty * FBX + tx + 1], dt16, F,
                                                          gp + gcol[r] - pitch - 1);
                if (GEN) {
                    if (xw[r])
                        tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, smm, skk, eo[r] - BX,
                                                              so[r] - PX, fo[ty * FBX + tx + 2], dt16, F,
                                                              gp + gcol[r] - pitch);
                    if (yw[r])
                        tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, smm, skk, eo[r] - 1,
                                                              so[r] - 1, fo[(ty + 1) * FBX + tx + 1], dt16, F,
                                                              gp + gcol[r] - 1);
                    if (xw[r] && yw[r])
                        tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, smm, skk, eo[r], so[r],
                                                              fo[(ty + 1) * FBX + tx + 2], dt16, F, gp + gcol[r]);
                }
            }
        }

        // prefetch psi for the next iteration: H at plane k+1, E at plane k
        fetch_psi((kw + 1 == nz) ? 0 : kw + 1, kw, true);
        // rotate stage, parity and H-ring slots
        if (s0 + 1 == S) par ^= 1u;
        s0 = s1;
        r2 = r1; r1 = r0; r0 = (r0 == 2) ? 0 : r0 + 1;
        kw = (kw + 1 == nz) ? 0 : kw + 1;
    }
    // drain: after an abort, wait (bounded) for the copies issued but never
    // waited for, so that no TMA write lands after the CTA has exited
    if (abort_flag) {
        if (tid == PRODUCER)
            for (int q = waited + 1; q < issued; ++q)
                if (q != withheld) mbar_wait_bounded(&bars[(gq0 + q) % S], uint32_t(((gq0 + q) / S) & 1));
        return -1;
    }
    return gq0 + Q;
}

// Class of a block: general (touches the CPML shell, a PEC wall or the last
// tile of an axis) or interior; an interior block also reports whether any of
// its cells (own or low halo) carries an antenna point (CTA-wide vote).
template <typename real, int TR, int R>
__device__ __forceinline__ void block_class(const StepArgs<real>& a, int i0, int j0, bool& gen, bool& src)
{
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    gen = i0 == 0 || j0 == 0 || i0 + 32 >= nx || j0 + TR >= ny ||
          (npml > 0 && (i0 - 1 < npml || i0 + 31 >= nx - npml || j0 - 1 < npml || j0 + TR - 1 >= ny - npml));
    src = false;
    if (!gen && a.smask) {
        constexpr int TW = TR / R;
        const int tx = threadIdx.x, tw = threadIdx.y;
        bool mine = false;
        #pragma unroll
        for (int r = 0; r < R; ++r) mine = mine || a.smask[(j0 + tw + r * TW) * nx + i0 + tx] != 0;
        if (tw == 0) mine = mine || a.smask[(j0 - 1) * nx + i0 + tx] != 0;
        if (tx == 0 && tw == 0)
            for (int jj = -1; jj < TR; ++jj) mine = mine || a.smask[(j0 + jj) * nx + i0 - 1] != 0;
        src = __syncthreads_or(mine) != 0;
    }
}

template <typename real, int TR, int R, int S>
__device__ __forceinline__ int tma_march_any(const StepArgs<real>& a, const TmaMaps& m, long long n, int i0, int j0,
                                             int kb, int ke, int* err, const MarchSmem<real, TR, S>& sm, int gq0)
{
    bool gen, src;
    block_class<real, TR, R>(a, i0, j0, gen, src);
    if (gen) return tma_march<real, TR, R, S, true, true>(a, m, n, i0, j0, kb, ke, err, sm, gq0);
    if (src) return tma_march<real, TR, R, S, false, true>(a, m, n, i0, j0, kb, ke, err, sm, gq0);
    return tma_march<real, TR, R, S, false, false>(a, m, n, i0, j0, kb, ke, err, sm, gq0);
}

template <typename real, int TR, int S>
__device__ __forceinline__ MarchSmem<real, TR, S> march_smem_init(int lz)
{
    using T = TmaTile<real, TR>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double tf[6];
    __shared__ int abort_flag;
    MarchSmem<real, TR, S> sm;
    sm.base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    sm.sH = reinterpret_cast<real*>(sm.base + S * T::STAGE);
    sm.uE = reinterpret_cast<Cpx<real>*>(sm.sH + 9 * T::P);
    sm.uH = sm.uE + (lz + 3);
    sm.bars = reinterpret_cast<uint64_t*>(sm.uH + (lz + 3));
    sm.tf = tf;
    sm.abort_flag = &abort_flag;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        abort_flag = 0;
        #pragma unroll 1
        for (int s = 0; s < S; ++s) mbar_init(&sm.bars[s], 1);
        mbar_fence_init();
    }
    return sm;
}

// Minimum resident CTAs per SM requested from the register allocator (the
// shared memory of a 32x8 FP32 tile fits three CTAs).
template <typename real, int TR, int R> struct MinCtas { static constexpr int value = 1; };
template <> struct MinCtas<float, 8, 1> { static constexpr int value = 3; };
template <> struct MinCtas<float, 8, 2> { static constexpr int value = 3; };
template <> struct MinCtas<float, 4, 1> { static constexpr int value = 4; };

// Grid: (ceil(nx/32), ceil(ny/TR), ceil(nz/lz)) CTAs of 32 x (TR/R) threads.
template <typename real, int TR, int R, int S>
__global__ void __launch_bounds__(32 * (TR / R), MinCtas<real, TR, R>::value)
yee_step_tma(const StepArgs<real> a, const __grid_constant__ TmaMaps m, long long n, int lz, int* err)
{
    const MarchSmem<real, TR, S> sm = march_smem_init<real, TR, S>(lz);
    const int kb = blockIdx.z * lz;
    tma_march_any<real, TR, R, S>(a, m, n, blockIdx.x * 32, blockIdx.y * TR, kb, min(kb + lz, a.nz), err, sm, 0);
}

}  // namespace fdtd
