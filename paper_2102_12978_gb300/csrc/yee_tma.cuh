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

template <typename real, int TY>
struct TmaTile {
    static constexpr int TX = 32;
    static constexpr int XA = 16 / int(sizeof(real));   // x alignment in elements
    static constexpr int BX = TX + 2 * XA;              // E / H box width
    static constexpr int EBY = TY + 2;                  // E box rows (j0-1 .. j0+TY)
    static constexpr int HBY = TY + 2;                  // H box rows (j0-1 .. j0+TY; the last row
                                                        // is read only at the +y wall, as zeros)
    static constexpr int FBX = TX + 2, FBY = TY + 1;    // fluence box (i0-2 .., j0-1 ..)
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t EB = al(size_t(BX) * EBY * sizeof(real));
    static constexpr size_t HB = al(size_t(BX) * HBY * sizeof(real));
    static constexpr size_t FB = al(size_t(FBX) * FBY * 8);
    static constexpr size_t STAGE = 3 * EB + 3 * HB + FB;
    static constexpr int PX = TX + 2, PY = TY + 2, P = PX * PY;   // H^{n+1/2} and H-bar rings
    static constexpr int NT = TX * TY;
    static constexpr int NHH = TX + TY + 1;
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

// |S| from |S|^2: FP64 grids take the correctly rounded square root; FP32
// grids take x * rsqrt(x) (a few ulp, far inside the FP32 tolerance of the
// fluence), which avoids the long correctly-rounded sequence per cell.
__device__ __forceinline__ double vec_norm(double x) { return sqrt(x); }
__device__ __forceinline__ float vec_norm(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

// Per-column constants of one H cell (own or halo): CPML shell membership,
// profile values, compact psi offsets, antenna mask.
template <typename real>
struct HCol {
    bool valid;
    int ci, cj;
    real chx, chy;
    bool xs, ys;
    real bx, ax, by, ay;
    int pxo, pyo;          // psi offsets within one plane of the x / y shell arrays
    uint8_t mk;
};

template <typename real, bool GEN, bool SRC>
__device__ __forceinline__ HCol<real> make_hcol(const StepArgs<real>& a, int ci, int cj)
{
    HCol<real> c;
    c.valid = ci >= 0 && ci < a.nx && cj >= 0 && cj < a.ny;
    if (!GEN) c.valid = ci != -1 || cj != -1;   // interior block: only "no cell" is invalid
    c.ci = ci; c.cj = cj;
    c.chx = real(0); c.chy = real(0); c.xs = false; c.ys = false;
    c.bx = c.ax = c.by = c.ay = real(0); c.pxo = c.pyo = 0; c.mk = 0;
    if (!c.valid) return c;
    c.chx = a.chx[ci]; c.chy = a.chy[cj];
    const int npml = a.npml, w2 = 2 * npml;
    if (GEN && npml > 0 && (ci < npml || ci >= a.nx - npml)) {
        const int ii = ci < npml ? ci : ci - a.nx + w2;
        c.xs = true; c.bx = a.bhx[ii]; c.ax = a.ahx[ii]; c.pxo = cj * w2 + ii;
    }
    if (GEN && npml > 0 && (cj < npml || cj >= a.ny - npml)) {
        const int jj = cj < npml ? cj : cj - a.ny + w2;
        c.ys = true; c.by = a.bhy[jj]; c.ay = a.ahy[jj]; c.pyo = jj * a.pitch + ci;
    }
    if (SRC && a.smask) c.mk = a.smask[cj * a.nx + ci];
    return c;
}

// H^{n+1/2} of one cell from the staged E planes k (e0*) and k+1 (e1*).
template <typename real, int BX, bool GEN, bool SRC>
__device__ __forceinline__ void tma_compute_h(const StepArgs<real>& a, const HCol<real>& c,
                                              const real* __restrict__ e0x, const real* __restrict__ e0y,
                                              const real* __restrict__ e0z, const real* __restrict__ e1x,
                                              const real* __restrict__ e1y, int idx, int kw, int psx_plane,
                                              int psy_plane, real& hx, real& hy, real& hz, Cpx<real> u,
                                              bool store, const real (&pp)[4])
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
    if (GEN && c.xs) {
        const int q = kw * psx_plane + c.pxo;
        const real p0 = c.bx * pp[0] + c.ax * dEz_x;   // Hyx (old value prefetched)
        const real p1 = c.bx * pp[1] + c.ax * dEy_x;   // Hzx
        hy += p0;
        hz -= p1;
        if (store) { a.phx_out[0][q] = p0; a.phx_out[1][q] = p1; }
    }
    if (GEN && c.ys) {
        const int q = kw * psy_plane + c.pyo;
        const real p0 = c.by * pp[2] + c.ay * dEz_y;   // Hxy
        const real p1 = c.by * pp[3] + c.ay * dEx_y;   // Hzy
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
template <typename real, int TY, int S>
struct MarchSmem {
    unsigned char* base;   // S stages
    real* sH;              // [3][3][P] ring of H^{n+1/2}
    Cpx<real>* uE;         // per-plane source factor at the E time, lz + 3 planes
    Cpx<real>* uH;         // the same at the H time
    uint64_t* bars;        // S mbarriers
    double* tf;            // 6 time factors
    int* abort_flag;
};

// One CTA marches one (32 x TY) x [kb, ke) block of a grid through one Yee
// step.  gq0 is the CTA's running plane counter (stage = gq % S, mbarrier
// parity = (gq / S) & 1), so that a persistent CTA can march many blocks
// with its mbarriers initialised once.  Returns the updated counter, or -1
// after a timed-out wait (the error word is raised).
// GEN: the block may touch the CPML shell, a PEC wall, the last (wall or
// ragged) tile of an axis; every per-cell check is compiled in.  !GEN: an
// interior block, where all of them are known false and compiled out.
// SRC: the block holds antenna cells (compiled out otherwise).
template <typename real, int TY, int S, bool GEN, bool SRC>
__device__ __forceinline__ int tma_march(const StepArgs<real>& a, const TmaMaps& m, long long n, int i0, int j0,
                                         int kb, int ke, int* err, const MarchSmem<real, TY, S>& sm, int gq0)
{
    static_assert(S >= 5, "the ring needs S >= 5 stages (lead of S-3 planes)");
    using T = TmaTile<real, TY>;
    using Acc = FluAcc<real>;
    using acc_t = typename Acc::T;
    constexpr int TX = T::TX, BX = T::BX, XA = T::XA, PX = T::PX, P = T::P, NT = T::NT, FBX = T::FBX;
    static_assert(T::NHH <= NT, "tile too small for its halo");
    unsigned char* base = sm.base;
    real* sH = sm.sH;
    uint64_t* bars = sm.bars;
    double* tf = sm.tf;
    int& abort_flag = *sm.abort_flag;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    constexpr int PRODUCER = (TY - 1) * 32;          // lane 0 of the last warp issues TMA
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    const int plane = pitch * ny;
    const int w2 = 2 * a.npml, psx_plane = ny * w2, psy_plane = w2 * pitch;
    const int i = i0 + tx, j = j0 + ty;
    const bool own = !GEN || ((i < nx) && (j < ny));
    const int so = (ty + 1) * PX + (tx + 1);        // own cell in the sH / sB rings
    const int eo = (ty + 1) * BX + (tx + XA);        // own cell in an E / H box
    const int gcol = j * pitch + i;
    const bool do_flu = a.fluence != nullptr;
    acc_t* F = static_cast<acc_t*>(a.fluence);
    const real dtr = real(a.dt);
    const int Q = ke - kb + 3;                       // E planes kb-1 .. ke+1

    auto stage = [&](int s) { return base + s * T::STAGE; };

    // ---- TMA producer (thread 0): plane q of this segment into stage q % S
    auto issue = [&](int q) {
        const int p = kb - 1 + q;
        const int pw = p < 0 ? p + nz : (p >= nz ? p - nz : p);
        const bool needH = p <= ke;
        const bool needF = do_flu && p >= kb && p <= ke - 1;
        const int s = (gq0 + q) % S;
        uint64_t* bar = &bars[s];
        unsigned char* st = stage(s);
        mbar_expect_tx(bar, 3 * T::E_BYTES + (needH ? 3 * T::H_BYTES : 0u) + (needF ? T::F_BYTES : 0u));
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
    // block, phase in FP64, stored in the field precision (read after the
    // first barrier of the march)
    if (SRC && a.smask) {
        for (int q = tid; q < Q; q += NT) {
            const int p = kb - 1 + q;
            const int pw = p < 0 ? p + nz : (p >= nz ? p - nz : p);
            const double2 z = a.zph[pw];
            // z (c - i s) f
            sm.uE[q].x = real((z.x * tf[0] + z.y * tf[1]) * tf[2]);
            sm.uE[q].y = real((z.y * tf[0] - z.x * tf[1]) * tf[2]);
            sm.uH[q].x = real((z.x * tf[3] + z.y * tf[4]) * tf[5]);
            sm.uH[q].y = real((z.y * tf[3] - z.x * tf[4]) * tf[5]);
        }
    }

    // per-column constants: own cell and this thread's H halo cell
    const HCol<real> co = make_hcol<real, GEN, SRC>(a, own ? i : -1, own ? j : -1);
    const real cex = own ? a.cex[i] : real(0), cey = own ? a.cey[j] : real(0);
    bool exs = false, eys = false;
    real ebx = 0, eax = 0, eby = 0, eay = 0;
    int epx = 0, epy = 0;
    if (GEN && own && w2 > 0) {
        if (i < a.npml || i >= nx - a.npml) {
            const int ii = i < a.npml ? i : i - nx + w2;
            exs = true; ebx = a.bex[ii]; eax = a.aex[ii]; epx = j * w2 + ii;
        }
        if (j < a.npml || j >= ny - a.npml) {
            const int jj = j < a.npml ? j : j - ny + w2;
            eys = true; eby = a.bey[jj]; eay = a.aey[jj]; epy = jj * pitch + i;
        }
    }
    // halo H cells: the row j0-1 on warp 0, the column i0-1 (TY+1 cells) on
    // warp TY/2, so that no warp carries both; the TMA producer is lane 0 of
    // warp TY-1
    int hs_h = 0, he_h = 0, hi_h = -1, hj_h = -1;
    if (ty == 0) { hi_h = i0 + tx; hj_h = j0 - 1; hs_h = tx + 1; he_h = tx + XA; }
    else if (ty == TY / 2 && tx <= TY) {
        const int jj = tx;
        hi_h = i0 - 1; hj_h = j0 - 1 + jj; hs_h = jj * PX; he_h = jj * BX + XA - 1;
    }
    const HCol<real> ch = make_hcol<real, GEN, SRC>(a, hi_h, hj_h);
    // fluence cells: base (i-1, j-1) and, in the last tiles, the wall cells
    const bool flu_base = !GEN || ((i >= 1) && (j >= 1) && (i <= nx) && (j <= ny));
    const bool xw = GEN && (tx == TX - 1) && (i == nx - 1) && (j >= 1) && (j <= ny);
    const bool yw = GEN && (ty == TY - 1) && (j == ny - 1) && (i >= 1) && (i <= nx);

    // CPML psi of the next plane, prefetched into registers one iteration ahead
    // (H side: own and halo cell, read copy; E side: own cell, updated in place)
    real ppo[4] = {0, 0, 0, 0}, pph[4] = {0, 0, 0, 0}, ppe[4] = {0, 0, 0, 0};
    auto fetch_psi_h = [&](const HCol<real>& c, int plane_w, real (&pp)[4]) {
        if (!GEN) return;
        if (c.xs) {
            const int q = plane_w * psx_plane + c.pxo;
            pp[0] = a.phx_in[0][q]; pp[1] = a.phx_in[1][q];
        }
        if (c.ys) {
            const int q = plane_w * psy_plane + c.pyo;
            pp[2] = a.phy_in[0][q]; pp[3] = a.phy_in[1][q];
        }
    };
    auto fetch_psi_e = [&](int plane_w) {
        if (!GEN) return;
        if (exs) { const int q = plane_w * psx_plane + epx; ppe[0] = a.pex[0][q]; ppe[1] = a.pex[1][q]; }
        if (eys) { const int q = plane_w * psy_plane + epy; ppe[2] = a.pey[0][q]; ppe[3] = a.pey[1][q]; }
    };
    {
        const int k0w = kb - 1 < 0 ? kb - 1 + nz : kb - 1;
        fetch_psi_h(co, k0w, ppo);
        fetch_psi_h(ch, k0w, pph);
    }

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
            constexpr int HS = int(T::HB / sizeof(real));
            real* hs = sH + r0 * 3 * P;
            const bool write_k = (k >= kb) && (k < ke);
            if (co.valid) {
                const real ox = hb[eo], oy = hb[HS + eo], oz = hb[2 * HS + eo];
                real hx = ox, hy = oy, hz = oz;
                tma_compute_h<real, BX, GEN, SRC>(a, co, e0x, e0y, e0z, e1x, e1y, eo, kw, psx_plane, psy_plane, hx, hy, hz,
                                        sm.uH[q], write_k, ppo);
                hs[so] = hx; hs[P + so] = hy; hs[2 * P + so] = hz;
                if (write_k) {
                    const int g = kw * plane + gcol;
                    a.hout[0][g] = hx; a.hout[1][g] = hy; a.hout[2][g] = hz;
                }
            }
            if (ch.valid) {
                const real ox = hb[he_h], oy = hb[HS + he_h], oz = hb[2 * HS + he_h];
                real hx = ox, hy = oy, hz = oz;
                tma_compute_h<real, BX, GEN, SRC>(a, ch, e0x, e0y, e0z, e1x, e1y, he_h, kw, psx_plane, psy_plane, hx, hy,
                                        hz, sm.uH[q], false, pph);
                hs[hs_h] = hx; hs[P + hs_h] = hy; hs[2 * P + hs_h] = hz;
            }
        }

        // ---- E^{n+1} of plane k-1 (needs H^{n+1/2} of planes k-1, k-2)
        const int km = k - 1;
        const int kmw = kw == 0 ? nz - 1 : kw - 1;
        const int sm1 = s0 == 0 ? S - 1 : s0 - 1;
        if (own && km >= kb && km < ke) {
            const real* h0 = sH + r1 * 3 * P;
            const real* h1 = sH + r2 * 3 * P;
            const unsigned char* stm = stage(sm1);
            const real ex = reinterpret_cast<const real*>(stm)[eo];
            const real ey = reinterpret_cast<const real*>(stm + T::EB)[eo];
            const real ez = reinterpret_cast<const real*>(stm + 2 * T::EB)[eo];
            const real hx0 = h0[so], hy0 = h0[P + so], hz0 = h0[2 * P + so];
            const real dHz_y = hz0 - h0[2 * P + so - PX];
            const real dHy_z = hy0 - h1[P + so];
            const real dHx_z = hx0 - h1[so];
            const real dHz_x = hz0 - h0[2 * P + so - 1];
            const real dHy_x = hy0 - h0[P + so - 1];
            const real dHx_y = hx0 - h0[so - PX];
            real nex = ex + cey * dHz_y - a.cz * dHy_z;
            real ney = ey + a.cz * dHx_z - cex * dHz_x;
            real nez = ez + cex * dHy_x - cey * dHx_y;
            if (GEN && exs) {
                const int qq = kmw * psx_plane + epx;
                const real p0 = ebx * ppe[0] + eax * dHz_x;   // Eyx (old value prefetched)
                const real p1 = ebx * ppe[1] + eax * dHy_x;   // Ezx
                a.pex[0][qq] = p0; a.pex[1][qq] = p1;
                ney -= p0;
                nez += p1;
            }
            if (GEN && eys) {
                const int qq = kmw * psy_plane + epy;
                const real p0 = eby * ppe[2] + eay * dHz_y;   // Exy
                const real p1 = eby * ppe[3] + eay * dHx_y;   // Ezy
                a.pey[0][qq] = p0; a.pey[1][qq] = p1;
                nex += p0;
                nez -= p1;
            }
            if (SRC && (co.mk & 0x07)) {
                const int ncol = nx * ny, col = j * nx + i;
                const Cpx<real>* B = static_cast<const Cpx<real>*>(a.scoefr);
                const Cpx<real> u = sm.uE[q - 1];
                if (co.mk & 0x01) { const Cpx<real> b = B[col]; nex += b.x * u.x - b.y * u.y; }
                if (co.mk & 0x02) { const Cpx<real> b = B[ncol + col]; ney += b.x * u.x - b.y * u.y; }
                if (co.mk & 0x04) { const Cpx<real> b = B[2 * ncol + col]; nez += b.x * u.x - b.y * u.y; }
            }
            if (GEN) {
                if (j == 0) { nex = real(0); nez = real(0); }    // PEC: tangential E
                if (i == 0) { ney = real(0); nez = real(0); }
            }
            const int g = kmw * plane + gcol;
            a.eout[0][g] = nex; a.eout[1][g] = ney; a.eout[2][g] = nez;
        }

        // ---- fluence of plane k-2: E planes k-2, k-1 and H-bar of k-2, k-1
        const int kf = k - 2;
        if (do_flu && kf >= kb && kf < ke && (flu_base || xw || yw)) {
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
            const real* sm = sH + r2 * 3 * P;
            const real* sk = sH + r1 * 3 * P;
            constexpr int HS = int(T::HB / sizeof(real));
            const real dt16 = dtr * real(0.0625);
            const int gp = kfw * plane;
            if (flu_base)
                tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, sm, sk, eo - BX - 1,
                                                      so - PX - 1, fo[ty * FBX + tx + 1], dt16, F,
                                                      gp + gcol - pitch - 1);
            if (xw)
                tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, sm, sk, eo - BX, so - PX,
                                                      fo[ty * FBX + tx + 2], dt16, F, gp + gcol - pitch);
            if (yw)
                tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, sm, sk, eo - 1, so - 1,
                                                      fo[(ty + 1) * FBX + tx + 1], dt16, F, gp + gcol - 1);
            if (xw && yw)
                tma_fluence_cell<real, BX, PX, P, HS>(emx, emy, emz, ekx, eky, hm, hk, sm, sk, eo, so,
                                                      fo[(ty + 1) * FBX + tx + 2], dt16, F, gp + gcol);
        }

        // prefetch psi for the next iteration: H at plane k+1, E at plane k
        {
            const int kn = (kw + 1 == nz) ? 0 : kw + 1;
            fetch_psi_h(co, kn, ppo);
            fetch_psi_h(ch, kn, pph);
            fetch_psi_e(kw);
        }
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
                mbar_wait_bounded(&bars[(gq0 + q) % S], uint32_t(((gq0 + q) / S) & 1));
        return -1;
    }
    return gq0 + Q;
}

// Class of a block: general (touches the CPML shell, a PEC wall or the last
// tile of an axis) or interior; an interior block also reports whether any of
// its cells (own or low halo) carries an antenna point (CTA-wide vote).
template <typename real, int TY>
__device__ __forceinline__ void block_class(const StepArgs<real>& a, int i0, int j0, bool& gen, bool& src)
{
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    gen = i0 == 0 || j0 == 0 || i0 + 32 >= nx || j0 + TY >= ny ||
          (npml > 0 && (i0 - 1 < npml || i0 + 31 >= nx - npml || j0 - 1 < npml || j0 + TY - 1 >= ny - npml));
    src = false;
    if (!gen && a.smask) {
        const int tx = threadIdx.x, ty = threadIdx.y;
        bool mine = a.smask[(j0 + ty) * nx + i0 + tx] != 0;
        if (ty == 0) mine = mine || a.smask[(j0 - 1) * nx + i0 + tx] != 0;
        if (tx == 0) mine = mine || a.smask[(j0 + ty) * nx + i0 - 1] != 0;
        if (tx == 0 && ty == 0) mine = mine || a.smask[(j0 - 1) * nx + i0 - 1] != 0;
        src = __syncthreads_or(mine) != 0;
    }
}

template <typename real, int TY, int S>
__device__ __forceinline__ int tma_march_any(const StepArgs<real>& a, const TmaMaps& m, long long n, int i0, int j0,
                                             int kb, int ke, int* err, const MarchSmem<real, TY, S>& sm, int gq0)
{
    bool gen, src;
    block_class<real, TY>(a, i0, j0, gen, src);
    if (gen) return tma_march<real, TY, S, true, true>(a, m, n, i0, j0, kb, ke, err, sm, gq0);
    if (src) return tma_march<real, TY, S, false, true>(a, m, n, i0, j0, kb, ke, err, sm, gq0);
    return tma_march<real, TY, S, false, false>(a, m, n, i0, j0, kb, ke, err, sm, gq0);
}

template <typename real, int TY, int S>
__device__ __forceinline__ MarchSmem<real, TY, S> march_smem_init(int lz)
{
    using T = TmaTile<real, TY>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double tf[6];
    __shared__ int abort_flag;
    MarchSmem<real, TY, S> sm;
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

// Minimum resident CTAs per SM requested from the register allocator: the
// FP32 32x8 tile fits three CTAs in shared memory, so cap its registers.
template <typename real, int TY> struct MinCtas { static constexpr int value = 1; };
template <> struct MinCtas<float, 8> { static constexpr int value = 3; };
template <> struct MinCtas<float, 4> { static constexpr int value = 4; };

template <typename real, int TY, int S>
__global__ void __launch_bounds__(32 * TY, MinCtas<real, TY>::value)
yee_step_tma(const StepArgs<real> a, const __grid_constant__ TmaMaps m, long long n, int lz, int* err)
{
    const MarchSmem<real, TY, S> sm = march_smem_init<real, TY, S>(lz);
    const int kb = blockIdx.z * lz;
    tma_march_any<real, TY, S>(a, m, n, blockIdx.x * 32, blockIdx.y * TY, kb, min(kb + lz, a.nz), err, sm, 0);
}

}  // namespace fdtd
