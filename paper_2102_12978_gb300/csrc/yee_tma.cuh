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
    static constexpr int HBY = TY + 1;                  // H box rows (j0-1 .. j0+TY-1)
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
    static constexpr size_t smem_bytes(int S) { return S * STAGE + 12 * size_t(P) * sizeof(real) + S * 8 + 128; }
};

// H^{n+1/2} of one cell from the staged planes (E of planes k and k+1 in
// box layout, H^{n-1/2} given); updates and optionally stores the H-side psi.
template <typename real, int BX>
__device__ __forceinline__ void tma_compute_h(const StepArgs<real>& a, const real* __restrict__ e0x,
                                              const real* __restrict__ e0y, const real* __restrict__ e0z,
                                              const real* __restrict__ e1x, const real* __restrict__ e1y,
                                              int idx, int ci, int cj, int kw, real hx, real hy, real hz,
                                              real chx, real chy, uint8_t mk, const double* tf, bool store,
                                              real& ohx, real& ohy, real& ohz)
{
    const real ex = e0x[idx], ey = e0y[idx], ez = e0z[idx];
    const real dEz_y = e0z[idx + BX] - ez;
    const real dEy_z = e1y[idx] - ey;
    const real dEx_z = e1x[idx] - ex;
    const real dEz_x = e0z[idx + 1] - ez;
    const real dEy_x = e0y[idx + 1] - ey;
    const real dEx_y = e0x[idx + BX] - ex;
    hx = hx - chy * dEz_y + a.cz * dEy_z;
    hy = hy - a.cz * dEx_z + chx * dEz_x;
    hz = hz - chx * dEy_x + chy * dEx_y;
    const int npml = a.npml, nx = a.nx, ny = a.ny;
    if (npml > 0) {
        const int w2 = 2 * npml;
        if (ci < npml || ci >= nx - npml) {
            const int ii = ci < npml ? ci : ci - nx + w2;
            const size_t q = (size_t(kw) * ny + cj) * w2 + ii;
            const real b = a.bhx[ii], aa = a.ahx[ii];
            const real p0 = b * a.phx_in[0][q] + aa * dEz_x;   // Hyx
            const real p1 = b * a.phx_in[1][q] + aa * dEy_x;   // Hzx
            hy += p0;
            hz -= p1;
            if (store) { a.phx_out[0][q] = p0; a.phx_out[1][q] = p1; }
        }
        if (cj < npml || cj >= ny - npml) {
            const int jj = cj < npml ? cj : cj - ny + w2;
            const size_t q = (size_t(kw) * w2 + jj) * a.pitch + ci;
            const real b = a.bhy[jj], aa = a.ahy[jj];
            const real p0 = b * a.phy_in[0][q] + aa * dEz_y;   // Hxy
            const real p1 = b * a.phy_in[1][q] + aa * dEx_y;   // Hzy
            hx -= p0;
            hz += p1;
            if (store) { a.phy_out[0][q] = p0; a.phy_out[1][q] = p1; }
        }
    }
    if (mk & 0x38) {
        const size_t ncol = size_t(nx) * ny, col = size_t(cj) * nx + ci;
        const double2 z = a.zph[kw];
        if (mk & 0x08) hx += real(source_value(a.scoef[3 * ncol + col], z, tf[3], tf[4], tf[5]));
        if (mk & 0x10) hy += real(source_value(a.scoef[4 * ncol + col], z, tf[3], tf[4], tf[5]));
        if (mk & 0x20) hz += real(source_value(a.scoef[5 * ncol + col], z, tf[3], tf[4], tf[5]));
    }
    ohx = hx; ohy = hy; ohz = hz;
}

template <typename real, int TY, int S>
__global__ void __launch_bounds__(32 * TY)
yee_step_tma(const StepArgs<real> a, const __grid_constant__ TmaMaps m, long long n, int lz, int* err)
{
    static_assert(S >= 4, "the ring needs S >= 4 stages (lead of S-2 planes)");
    using T = TmaTile<real, TY>;
    constexpr int TX = T::TX, BX = T::BX, XA = T::XA, PX = T::PX, P = T::P, NT = T::NT, FBX = T::FBX;
    static_assert(T::NHH <= NT, "tile too small for its halo");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    real* sH = reinterpret_cast<real*>(base + S * T::STAGE);   // [2][3][P]
    real* sB = sH + 6 * P;                                      // [2][3][P]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + 6 * P);
    __shared__ double tf[6];
    __shared__ int abort_flag;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int kb = blockIdx.z * lz;
    const int ke = min(kb + lz, a.nz);
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch, npml = a.npml;
    const size_t plane = size_t(pitch) * ny;
    const int i = i0 + tx, j = j0 + ty;
    const bool own = (i < nx) && (j < ny);
    const int so = (ty + 1) * PX + (tx + 1);        // own cell in the sH / sB rings
    const int eo = (ty + 1) * BX + (tx + XA);        // own cell in an E / H box
    const bool do_flu = a.fluence != nullptr;
    const int Q = ke - kb + 3;                       // planes kb-1 .. ke+1

    auto stage = [&](int q) { return base + (q % S) * T::STAGE; };
    auto Ebox = [&](int q, int c) { return reinterpret_cast<real*>(stage(q) + c * T::EB); };
    auto Hbox = [&](int q, int c) { return reinterpret_cast<real*>(stage(q) + 3 * T::EB + c * T::HB); };
    auto Fbox = [&](int q) { return reinterpret_cast<double*>(stage(q) + 3 * T::EB + 3 * T::HB); };

    auto issue = [&](int q) {
        const int p = kb - 1 + q;
        const int pw = ((p % nz) + nz) % nz;
        const bool needH = p <= ke;
        const bool needF = do_flu && p >= kb && p <= ke - 1;
        uint64_t* bar = &bars[q % S];
        mbar_expect_tx(bar, 3 * T::E_BYTES + (needH ? 3 * T::H_BYTES : 0u) + (needF ? T::F_BYTES : 0u));
        #pragma unroll
        for (int c = 0; c < 3; ++c) tma_load_3d(Ebox(q, c), &m.e[c], bar, i0 - XA, j0 - 1, pw);
        if (needH) {
            #pragma unroll
            for (int c = 0; c < 3; ++c) tma_load_3d(Hbox(q, c), &m.h[c], bar, i0 - XA, j0 - 1, pw);
        }
        if (needF) tma_load_3d(Fbox(q), &m.f, bar, i0 - 2, j0 - 1, pw);
    };

    int issued = 0;
    if (tid == 0) {
        abort_flag = 0;
        #pragma unroll 1
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
        double c, s, f;
        source_time(a.st, (double(n) + 0.5) * a.dt, c, s, f);
        tf[3] = c; tf[4] = s; tf[5] = f;
        source_time(a.st, (double(n) + 1.0) * a.dt, c, s, f);
        tf[0] = c; tf[1] = s; tf[2] = f;
    }
    for (int q = tid; q < 12 * P; q += NT) sH[q] = real(0);   // sH and sB
    __syncthreads();
    if (tid == 0) {
        for (; issued < S - 2 && issued < Q; ++issued) issue(issued);
    }

    // H halo cell of this thread: row j0-1 (tid < TX) or column i0-1
    int hi_h = -1, hj_h = -1, hs_h = 0, he_h = 0;
    if (tid < T::NHH) {
        if (tid < TX) { hi_h = i0 + tid; hj_h = j0 - 1; hs_h = tid + 1; he_h = tid + XA; }
        else {
            const int jj = tid - TX;
            hi_h = i0 - 1; hj_h = j0 - 1 + jj; hs_h = jj * PX; he_h = jj * BX + XA - 1;
        }
    }
    const bool halo_h_in = hi_h >= 0 && hi_h < nx && hj_h >= 0 && hj_h < ny;
    const uint8_t mk_own = (own && a.smask) ? a.smask[size_t(j) * nx + i] : uint8_t(0);
    const uint8_t mk_hh = (halo_h_in && a.smask) ? a.smask[size_t(hj_h) * nx + hi_h] : uint8_t(0);
    const real chx_o = own ? a.chx[i] : real(0), chy_o = own ? a.chy[j] : real(0);
    const real cex_o = own ? a.cex[i] : real(0), cey_o = own ? a.cey[j] : real(0);
    const real chx_h = halo_h_in ? a.chx[hi_h] : real(0), chy_h = halo_h_in ? a.chy[hj_h] : real(0);
    const bool xw = (tx == TX - 1) && (i == nx - 1);
    const bool yw = (ty == TY - 1) && (j == ny - 1);

    int waited = -1;   // highest plane this thread has seen complete
    #pragma unroll 1
    for (int q = 0; q <= Q - 2; ++q) {
        const int k = kb - 1 + q;
        bool ok = true;
        if (q == 0) ok = mbar_wait_bounded(&bars[0], 0);
        ok = ok && mbar_wait_bounded(&bars[(q + 1) % S], uint32_t(((q + 1) / S) & 1));
        if (ok) waited = q + 1;
        else { abort_flag = 1; atomicOr(err, 1); }
        __syncthreads();   // A: planes k, k+1 landed; readers of plane k-2's stage done
        if (abort_flag) break;
        if (tid == 0 && issued < Q) { fence_proxy_async(); issue(issued); ++issued; }

        const int kw = ((k % nz) + nz) % nz;
        const bool write_k = (k >= kb) && (k < ke);
        const real* e0x = Ebox(q, 0); const real* e0y = Ebox(q, 1); const real* e0z = Ebox(q, 2);
        const real* e1x = Ebox(q + 1, 0); const real* e1y = Ebox(q + 1, 1);
        const real* hbx = Hbox(q, 0); const real* hby = Hbox(q, 1); const real* hbz = Hbox(q, 2);
        real* hs = sH + (k & 1) * 3 * P;
        real* bs = sB + (k & 1) * 3 * P;
        if (own) {
            const real ox = hbx[eo], oy = hby[eo], oz = hbz[eo];
            real nxh, nyh, nzh;
            tma_compute_h<real, BX>(a, e0x, e0y, e0z, e1x, e1y, eo, i, j, kw, ox, oy, oz, chx_o, chy_o,
                                    mk_own, tf, write_k, nxh, nyh, nzh);
            hs[so] = nxh; hs[P + so] = nyh; hs[2 * P + so] = nzh;
            bs[so] = real(0.5) * (ox + nxh); bs[P + so] = real(0.5) * (oy + nyh);
            bs[2 * P + so] = real(0.5) * (oz + nzh);
            if (write_k) {
                const size_t g = size_t(kw) * plane + size_t(j) * pitch + i;
                a.hout[0][g] = nxh; a.hout[1][g] = nyh; a.hout[2][g] = nzh;
            }
        } else {
            hs[so] = real(0); hs[P + so] = real(0); hs[2 * P + so] = real(0);
            bs[so] = real(0); bs[P + so] = real(0); bs[2 * P + so] = real(0);
        }
        if (tid < T::NHH) {
            if (halo_h_in) {
                const real ox = hbx[he_h], oy = hby[he_h], oz = hbz[he_h];
                real nxh, nyh, nzh;
                tma_compute_h<real, BX>(a, e0x, e0y, e0z, e1x, e1y, he_h, hi_h, hj_h, kw, ox, oy, oz, chx_h,
                                        chy_h, mk_hh, tf, false, nxh, nyh, nzh);
                hs[hs_h] = nxh; hs[P + hs_h] = nyh; hs[2 * P + hs_h] = nzh;
                bs[hs_h] = real(0.5) * (ox + nxh); bs[P + hs_h] = real(0.5) * (oy + nyh);
                bs[2 * P + hs_h] = real(0.5) * (oz + nzh);
            } else {
                hs[hs_h] = real(0); hs[P + hs_h] = real(0); hs[2 * P + hs_h] = real(0);
                bs[hs_h] = real(0); bs[P + hs_h] = real(0); bs[2 * P + hs_h] = real(0);
            }
        }
        __syncthreads();   // B: H^{n+1/2} of planes k, k-1 and H-bar visible

        if (write_k && own) {
            const real* h0 = sH + (k & 1) * 3 * P;
            const real* h1 = sH + ((k - 1) & 1) * 3 * P;
            const real ex = e0x[eo], ey = e0y[eo], ez = e0z[eo];
            const real hx0 = h0[so], hy0 = h0[P + so], hz0 = h0[2 * P + so];
            const real dHz_y = hz0 - h0[2 * P + so - PX];
            const real dHy_z = hy0 - h1[P + so];
            const real dHx_z = hx0 - h1[so];
            const real dHz_x = hz0 - h0[2 * P + so - 1];
            const real dHy_x = hy0 - h0[P + so - 1];
            const real dHx_y = hx0 - h0[so - PX];
            real nex = ex + cey_o * dHz_y - a.cz * dHy_z;
            real ney = ey + a.cz * dHx_z - cex_o * dHz_x;
            real nez = ez + cex_o * dHy_x - cey_o * dHx_y;
            if (npml > 0) {
                const int w2 = 2 * npml;
                if (i < npml || i >= nx - npml) {
                    const int ii = i < npml ? i : i - nx + w2;
                    const size_t qq = (size_t(kw) * ny + j) * w2 + ii;
                    const real b = a.bex[ii], aa = a.aex[ii];
                    const real p0 = b * a.pex[0][qq] + aa * dHz_x;   // Eyx
                    const real p1 = b * a.pex[1][qq] + aa * dHy_x;   // Ezx
                    a.pex[0][qq] = p0; a.pex[1][qq] = p1;
                    ney -= p0;
                    nez += p1;
                }
                if (j < npml || j >= ny - npml) {
                    const int jj = j < npml ? j : j - ny + w2;
                    const size_t qq = (size_t(kw) * w2 + jj) * pitch + i;
                    const real b = a.bey[jj], aa = a.aey[jj];
                    const real p0 = b * a.pey[0][qq] + aa * dHz_y;   // Exy
                    const real p1 = b * a.pey[1][qq] + aa * dHx_y;   // Ezy
                    a.pey[0][qq] = p0; a.pey[1][qq] = p1;
                    nex += p0;
                    nez -= p1;
                }
            }
            if (mk_own & 0x07) {
                const size_t ncol = size_t(nx) * ny, col = size_t(j) * nx + i;
                const double2 z = a.zph[kw];
                if (mk_own & 0x01) nex += real(source_value(a.scoef[col], z, tf[0], tf[1], tf[2]));
                if (mk_own & 0x02) ney += real(source_value(a.scoef[ncol + col], z, tf[0], tf[1], tf[2]));
                if (mk_own & 0x04) nez += real(source_value(a.scoef[2 * ncol + col], z, tf[0], tf[1], tf[2]));
            }
            if (j == 0) { nex = real(0); nez = real(0); }    // PEC: tangential E
            if (i == 0) { ney = real(0); nez = real(0); }
            const size_t g = size_t(kw) * plane + size_t(j) * pitch + i;
            a.eout[0][g] = nex; a.eout[1][g] = ney; a.eout[2][g] = nez;
        }

        if (do_flu && k >= kb + 1) {
            // cells (fi, fj, k-1), fi in {i-1, i at the +x wall}, fj likewise
            const int km = k - 1;
            const int kmw = ((km % nz) + nz) % nz;
            const real* emx = Ebox(q - 1, 0); const real* emy = Ebox(q - 1, 1); const real* emz = Ebox(q - 1, 2);
            const real* ekx = e0x; const real* eky = e0y;
            const real* bm = sB + (km & 1) * 3 * P;
            const real* bk = sB + (k & 1) * 3 * P;
            using Acc = FluAcc<real>;
            const typename Acc::T* fo = reinterpret_cast<const typename Acc::T*>(Fbox(q - 1));
            typename Acc::T* F = static_cast<typename Acc::T*>(a.fluence);
            const real dtr = real(a.dt);
            #pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const int di = qq & 1, dj = qq >> 1;
                if (di && !xw) continue;
                if (dj && !yw) continue;
                const int fi = i - 1 + di, fj = j - 1 + dj;
                if (fi < 0 || fj < 0 || fi >= nx || fj >= ny) continue;
                const int ce = eo - BX - 1 + dj * BX + di;      // E box index of (fi, fj)
                const int cs = so - PX - 1 + dj * PX + di;      // sB index of (fi, fj)
                const int cf = (ty + dj) * FBX + (tx + 1 + di); // fluence box index of (fi, fj)
                const real ex = real(0.25) * (emx[ce] + emx[ce + BX] + ekx[ce] + ekx[ce + BX]);
                const real ey = real(0.25) * (emy[ce] + emy[ce + 1] + eky[ce] + eky[ce + 1]);
                const real ez = real(0.25) * (emz[ce] + emz[ce + 1] + emz[ce + BX] + emz[ce + BX + 1]);
                const real hx = real(0.5) * (bm[cs] + bm[cs + 1]);
                const real hy = real(0.5) * (bm[P + cs] + bm[P + cs + PX]);
                const real hz = real(0.5) * (bm[2 * P + cs] + bk[2 * P + cs]);
                const real sx = ey * hz - ez * hy;
                const real sy = ez * hx - ex * hz;
                const real sz = ex * hy - ey * hx;
                const real sm = sqrt(sx * sx + sy * sy + sz * sz);
                const size_t g = size_t(kmw) * plane + size_t(fj) * pitch + fi;
                F[g] = Acc::add(fo[cf], sm * dtr);
            }
        }
    }
    // drain: after an abort, wait (bounded) for the copies issued but never
    // waited for, so that no TMA write lands after the CTA has exited
    if (tid == 0 && abort_flag) {
        for (int q = waited + 1; q < issued; ++q) mbar_wait_bounded(&bars[q % S], uint32_t((q / S) & 1));
    }
}

}  // namespace fdtd
