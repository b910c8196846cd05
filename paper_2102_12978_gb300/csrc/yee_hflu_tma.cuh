// yee_hflu_tma.cuh -- H pass of the two-pass Yee step with the fluence term
// (sm_103a, TMA-staged).
//
// Pass 1 of a step: H^{n-1/2} -> H^{n+1/2} (curl of E^n, CPML psi of the H
// side, soft source at (n+1/2) dt; Section 4, Eq. 13) and the fluence term
// |E^n_c x Hbar^n_c| dt of every cell (Section 2), Hbar = (H^{n-1/2} +
// H^{n+1/2}) / 2.  Pass 2 (e_column in yee_split.cuh, without its fluence
// part) then takes E^n -> E^{n+1}.
//
// A CTA of 32 x TY threads owns a 32 x TY tile of columns and marches the z
// planes kb .. ke of its segment.  One thread issues cp.async.bulk.tensor.3d
// box loads of each plane -- E^n and H^{n-1/2} over the tile plus one cell
// on the +x and +y sides, and the old fluence of the tile -- into an
// S-stage shared-memory ring, S-2 planes ahead of use; each stage completes
// on its own mbarrier.  Box elements past nx / ny read as zeros, the virtual
// wall value.  In iteration k the CTA computes H^{n+1/2} of plane k and the
// fluence of plane k-1, whose cell centre needs H^{n+1/2} of planes k-1
// (the four faces around it) and k (Hz above it):
//   * own-cell H^{n+1/2} of plane k-1 and Hz of plane k are the thread's own
//     registers;
//   * Hx at i+1 and Hy at j+1 come from a two-slot shared exchange written in
//     the previous iteration; the tile's +x column of Hx and +y row of Hy are
//     computed (not stored) by warp 0 and the last warp;
//   * the last plane ke is computed for Hz only (the next segment stores it).
// Every wait is bounded; on expiry the CTA raises the grid's error word,
// drains its own copies and returns.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "yee_fused.cuh"
#include "yee_tma.cuh"

namespace fdtd {

template <typename real, int TY>
struct HFluTile {
    static constexpr int TX = 32;
    static constexpr int XA = 16 / int(sizeof(real));
    static constexpr int BX = (TX + 1 + XA - 1) / XA * XA;   // columns i0 .. i0+BX-1 (>= i0+32)
    static constexpr int BY = TY + 1;                        // rows j0 .. j0+TY
    static constexpr int FBX = TX, FBY = TY;                 // fluence box (8-byte cells)
    static constexpr size_t al(size_t v) { return (v + 127) / 128 * 128; }
    static constexpr size_t B = al(size_t(BX) * BY * sizeof(real));
    static constexpr size_t FB = al(size_t(FBX) * FBY * 8);
    static constexpr size_t STAGE = 6 * B + FB;              // E (3), H^{n-1/2} (3), fluence
    static constexpr uint32_t BOX_BYTES = uint32_t(BX * BY * sizeof(real));
    static constexpr uint32_t F_BYTES = uint32_t(FBX * FBY * 8);
    static constexpr int XH = (TX + 1) * TY;                 // exchange: Hx of columns i0 .. i0+32
    static constexpr int YH = TX * (TY + 1);                 //           Hy of rows j0 .. j0+TY
    static constexpr int XS = XH + YH;
    // stages + two exchange slots + per-plane source factors + mbarriers
    static constexpr size_t smem_bytes(int S, int lz)
    {
        return S * STAGE + 2 * size_t(XS) * sizeof(real) + size_t(lz + 2) * 2 * sizeof(real) + S * 8 + 128;
    }
};

// H^{n+1/2} components of one cell (mask: which components to compute) from
// the staged E planes k (e0*) and k+1 (e1*) at box index idx and the old H
// values; x/y shell psi read from the read copy and, if `store`, written to
// the write copy.  ci / cj: the cell; ii / jj: shell indices or -1.
// chx / chy: the cell's curl coefficients.  Only the box elements the
// selected components need are read (the +y row of the Hy halo has no row
// above it in the box).
template <typename real, int BX, bool GEN, bool SRC, int COMP>
__device__ __forceinline__ void hflu_cell(const StepArgs<real>& a, int ci, int cj, int ii, int jj, int kw, real chx,
                                          real chy, const real* __restrict__ e0x, const real* __restrict__ e0y,
                                          const real* __restrict__ e0z, const real* __restrict__ e1x,
                                          const real* __restrict__ e1y, int idx, real& hx, real& hy, real& hz,
                                          uint8_t mk, Cpx<real> u, bool store)
{
    constexpr bool X = COMP & 1, Y = COMP & 2, Z = COMP & 4;
    const real ex = e0x[idx], ey = e0y[idx];
    real ez = real(0), dEz_y = real(0), dEz_x = real(0), dEy_x = real(0), dEx_y = real(0);
    if (X || Y) ez = e0z[idx];
    if (X) dEz_y = e0z[idx + BX] - ez;
    if (Y) dEz_x = e0z[idx + 1] - ez;
    if (Z) dEy_x = e0y[idx + 1] - ey;
    if (Z) dEx_y = e0x[idx + BX] - ex;
    if (X) hx = hx - chy * dEz_y + a.cz * (e1y[idx] - ey);
    if (Y) hy = hy - a.cz * (e1x[idx] - ex) + chx * dEz_x;
    if (Z) hz = hz - chx * dEy_x + chy * dEx_y;
    const int w2 = 2 * a.npml;
    if (GEN && ii >= 0 && (Y || Z)) {
        const int q = (kw * a.ny + cj) * w2 + ii;
        const real b = a.bhx[ii], aa = a.ahx[ii];
        if (Y) {
            const real p0 = b * a.phx_in[0][q] + aa * dEz_x;   // Hyx
            hy += p0;
            if (store) a.phx_out[0][q] = p0;
        }
        if (Z) {
            const real p1 = b * a.phx_in[1][q] + aa * dEy_x;   // Hzx
            hz -= p1;
            if (store) a.phx_out[1][q] = p1;
        }
    }
    if (GEN && jj >= 0 && (X || Z)) {
        const int q = (kw * w2 + jj) * a.pitch + ci;
        const real b = a.bhy[jj], aa = a.ahy[jj];
        if (X) {
            const real p0 = b * a.phy_in[0][q] + aa * dEz_y;   // Hxy
            hx -= p0;
            if (store) a.phy_out[0][q] = p0;
        }
        if (Z) {
            const real p1 = b * a.phy_in[1][q] + aa * dEx_y;   // Hzy
            hz += p1;
            if (store) a.phy_out[1][q] = p1;
        }
    }
    if (SRC && (mk & 0x38)) {
        const int ncol = a.nx * a.ny, col = cj * a.nx + ci;
        const Cpx<real>* Bc = static_cast<const Cpx<real>*>(a.scoefr);
        if (X && (mk & 0x08)) { const Cpx<real> b = Bc[3 * ncol + col]; hx += b.x * u.x - b.y * u.y; }
        if (Y && (mk & 0x10)) { const Cpx<real> b = Bc[4 * ncol + col]; hy += b.x * u.x - b.y * u.y; }
        if (Z && (mk & 0x20)) { const Cpx<real> b = Bc[5 * ncol + col]; hz += b.x * u.x - b.y * u.y; }
    }
}

// Class of an H-pass block: gen = it needs the wall / ragged / CPML checks
// (its cells or its +x / +y halo reach a wall, a ragged edge or the shell);
// src = (interior) its cells or halo hold antenna points.  Block-uniform.
template <typename real, int TY>
__device__ __forceinline__ void hflu_class(const StepArgs<real>& a, int i0, int j0, bool& gen, bool& src)
{
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    gen = i0 + 32 >= nx || j0 + TY >= ny ||
          (npml > 0 && (i0 < npml || i0 + 32 >= nx - npml || j0 < npml || j0 + TY >= ny - npml));
    src = false;
    if (!gen && a.smask) {
        const int tx = threadIdx.x, ty = threadIdx.y;
        bool mine = a.smask[(j0 + ty) * nx + i0 + tx] != 0;
        if (ty == 0 && tx < TY) mine = mine || a.smask[(j0 + tx) * nx + i0 + 32] != 0;
        if (ty == TY - 1) mine = mine || a.smask[(j0 + TY) * nx + i0 + tx] != 0;
        src = __syncthreads_or(mine) != 0;
    }
}

template <typename real, int TY, int S, bool GEN, bool SRC>
__device__ __forceinline__ void hflu_march(const StepArgs<real>& a, const TmaMaps& m, long long n, int i0, int j0,
                                           int kb, int ke, int* err, unsigned char* base, real* xs,
                                           Cpx<real>* uH, uint64_t* bars, double* tf, int& abort_flag)
{
    static_assert(S >= 4, "the ring needs S >= 4 stages");
    using T = HFluTile<real, TY>;
    using Acc = FluAcc<real>;
    using acc_t = typename Acc::T;
    constexpr int BX = T::BX, XH = T::XH, XS = T::XS, NT = 32 * TY;
    constexpr int PRODUCER = (TY - 1) * 32;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch, plane = pitch * ny;
    const int i = i0 + tx, j = j0 + ty;
    const bool do_flu = a.fluence != nullptr;
    acc_t* F = static_cast<acc_t*>(a.fluence);
    const int Q = ke - kb + 1;   // planes kb .. ke (ke wrapped)

    auto stage = [&](int s) { return base + s * T::STAGE; };
    auto issue = [&](int q) {
        const int p = kb + q;
        const int pw = p >= nz ? p - nz : p;
        const bool needF = do_flu && q < Q - 1;
        const int s = q % S;
        uint64_t* bar = &bars[s];
        unsigned char* st = stage(s);
        mbar_expect_tx(bar, 6 * T::BOX_BYTES + (needF ? T::F_BYTES : 0u));
        #pragma unroll
        for (int c = 0; c < 3; ++c) tma_load_3d(st + c * T::B, &m.e[c], bar, i0, j0, pw);
        #pragma unroll
        for (int c = 0; c < 3; ++c) tma_load_3d(st + (3 + c) * T::B, &m.h[c], bar, i0, j0, pw);
        if (needF) tma_load_3d(st + 6 * T::B, &m.f, bar, i0, j0, pw);
    };

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        mbar_fence_init();
        double c, s, f;
        source_time(a.st, (double(n) + 0.5) * a.dt, c, s, f);
        tf[0] = c; tf[1] = s; tf[2] = f;
    }
    __syncthreads();
    int issued = 0;
    if (tid == PRODUCER) {
        #pragma unroll 1
        for (; issued < S - 2 && issued < Q; ++issued) issue(issued);
    }
    if (SRC && a.smask) {
        for (int q = tid; q < Q; q += NT) {
            const int p = kb + q;
            const double2 z = a.zph[p >= nz ? p - nz : p];
            uH[q].x = real((z.x * tf[0] + z.y * tf[1]) * tf[2]);
            uH[q].y = real((z.y * tf[0] - z.x * tf[1]) * tf[2]);
        }
    }

    // ---- per-cell constants
    const bool own = !GEN || (i < nx && j < ny);
    const int npml = a.npml, w2 = 2 * npml;
    auto shell_x = [&](int c) { return (GEN && npml > 0 && c >= 0 && (c < npml || c >= nx - npml)) ? (c < npml ? c : c - nx + w2) : -1; };
    auto shell_y = [&](int c) { return (GEN && npml > 0 && c >= 0 && (c < npml || c >= ny - npml)) ? (c < npml ? c : c - ny + w2) : -1; };
    const int ii = own ? shell_x(i) : -1, jj = own ? shell_y(j) : -1;
    const uint8_t mk = (SRC && a.smask && own) ? a.smask[j * nx + i] : uint8_t(0);
    const real chx = own ? a.chx[i] : real(0), chy = own ? a.chy[j] : real(0);
    const int bo = ty * BX + tx;          // own cell in the boxes
    const int gcol = j * pitch + i;
    // halo cells: Hx of column i0+32 (warp 0, lanes < TY) and Hy of row j0+TY
    // (last warp, all lanes)
    const bool hxh = ty == 0 && tx < TY;
    const bool hyh = ty == TY - 1;
    int hci = 0, hcj = 0, hbo = 0, hii = -1, hjj = -1;
    bool hval = false;
    uint8_t hmk = 0;
    real hchx = real(0), hchy = real(0);
    if (hxh) { hci = i0 + 32; hcj = j0 + tx; hbo = tx * BX + 32; }
    if (hyh) { hci = i0 + tx; hcj = j0 + TY; hbo = TY * BX + tx; }
    if (hxh || hyh) {
        hval = !GEN || (hci < nx && hcj < ny);
        if (hval) {
            hii = shell_x(hci); hjj = shell_y(hcj);
            hchx = a.chx[hci]; hchy = a.chy[hcj];
            if (SRC && a.smask) hmk = a.smask[hcj * nx + hci];
        }
    }
    const real dt16 = real(a.dt16);

    real px = real(0), py = real(0), pz = real(0);   // own H^{n+1/2} of the previous plane
    int waited = -1;
    #pragma unroll 1
    for (int q = 0; q < Q; ++q) {
        const int k = kb + q;
        const int kw = k >= nz ? k - nz : k;
        const int s0 = q % S, s1 = (q + 1) % S;
        bool ok = true;
        if (q == 0) ok = mbar_wait_bounded(&bars[s0], 0u);
        if (q + 1 < Q) ok = ok && mbar_wait_bounded(&bars[s1], uint32_t(((q + 1) / S) & 1));
        if (ok) waited = q + 1;
        else { abort_flag = 1; atomicOr(err, 1); }
        __syncthreads();   // planes q, q+1 landed; every reader of plane q-2 and slot q&1 is done
        if (abort_flag) break;
        if (tid == PRODUCER && issued < Q) { fence_proxy_async(); issue(issued); ++issued; }

        const unsigned char* st0 = stage(s0);
        const unsigned char* st1 = stage(s1);
        const real* e0x = reinterpret_cast<const real*>(st0);
        const real* e0y = reinterpret_cast<const real*>(st0 + T::B);
        const real* e0z = reinterpret_cast<const real*>(st0 + 2 * T::B);
        const real* o0x = reinterpret_cast<const real*>(st0 + 3 * T::B);
        const real* o0y = reinterpret_cast<const real*>(st0 + 4 * T::B);
        const real* o0z = reinterpret_cast<const real*>(st0 + 5 * T::B);
        const real* e1x = reinterpret_cast<const real*>(st1);
        const real* e1y = reinterpret_cast<const real*>(st1 + T::B);
        Cpx<real> u;
        if (SRC) u = uH[q];
        real* xw = xs + (q & 1) * XS;             // exchange slot of plane k
        const bool last = q == Q - 1;

        // ---- H^{n+1/2} of plane k (only Hz on the last plane)
        real hx = o0x[bo], hy = o0y[bo], hz = o0z[bo];
        if (!last) {
            if (own) {
                hflu_cell<real, BX, GEN, SRC, 7>(a, i, j, ii, jj, kw, chx, chy, e0x, e0y, e0z, e1x, e1y, bo, hx, hy,
                                                 hz, mk, u, true);
                const int g = kw * plane + gcol;
                a.hout[0][g] = hx; a.hout[1][g] = hy; a.hout[2][g] = hz;
            } else {
                hx = hy = hz = real(0);
            }
            xw[ty * 33 + tx] = hx;                // Hx exchange [TY][33]
            xw[XH + ty * 32 + tx] = hy;           // Hy exchange [TY+1][32]
            if (hxh) {
                real v = real(0), d1 = real(0), d2 = real(0);
                if (hval) {
                    v = o0x[hbo];
                    hflu_cell<real, BX, GEN, SRC, 1>(a, hci, hcj, hii, hjj, kw, hchx, hchy, e0x, e0y, e0z, e1x, e1y,
                                                     hbo, v, d1, d2, hmk, u, false);
                }
                xw[tx * 33 + 32] = v;
            }
            if (hyh) {
                real v = real(0), d1 = real(0), d2 = real(0);
                if (hval) {
                    v = o0y[hbo];
                    hflu_cell<real, BX, GEN, SRC, 2>(a, hci, hcj, hii, hjj, kw, hchx, hchy, e0x, e0y, e0z, e1x, e1y,
                                                     hbo, d1, v, d2, hmk, u, false);
                }
                xw[XH + TY * 32 + tx] = v;
            }
        } else if (own) {
            real d1 = real(0), d2 = real(0);
            hflu_cell<real, BX, GEN, SRC, 4>(a, i, j, ii, jj, kw, chx, chy, e0x, e0y, e0z, e1x, e1y, bo, d1, d2, hz, mk,
                                             u, false);
        } else {
            hz = real(0);
        }

        // ---- fluence of plane k-1: E^n of planes k-1, k; Hbar of planes k-1, k
        if (do_flu && q >= 1 && own) {
            const int sm1 = (q - 1) % S;
            const unsigned char* stm = stage(sm1);
            const real* mx = reinterpret_cast<const real*>(stm);
            const real* my = reinterpret_cast<const real*>(stm + T::B);
            const real* mz = reinterpret_cast<const real*>(stm + 2 * T::B);
            const real* omx = reinterpret_cast<const real*>(stm + 3 * T::B);
            const real* omy = reinterpret_cast<const real*>(stm + 4 * T::B);
            const real* omz = reinterpret_cast<const real*>(stm + 5 * T::B);
            const acc_t* fo = reinterpret_cast<const acc_t*>(stm + 6 * T::B);
            const real* xr = xs + ((q - 1) & 1) * XS;   // exchange slot of plane k-1
            const real cx = (mx[bo] + mx[bo + BX]) + (e0x[bo] + e0x[bo + BX]);
            const real cy = (my[bo] + my[bo + 1]) + (e0y[bo] + e0y[bo + 1]);
            const real cz = (mz[bo] + mz[bo + 1]) + (mz[bo + BX] + mz[bo + BX + 1]);
            const real hbx = (omx[bo] + px) + (omx[bo + 1] + xr[ty * 33 + tx + 1]);
            const real hby = (omy[bo] + py) + (omy[bo + BX] + xr[XH + (ty + 1) * 32 + tx]);
            const real hbz = (omz[bo] + pz) + (o0z[bo] + hz);
            const real sx = cy * hbz - cz * hby;
            const real sy = cz * hbx - cx * hbz;
            const real sz = cx * hby - cy * hbx;
            const int kf = kw == 0 ? nz - 1 : kw - 1;
            F[kf * plane + gcol] = Acc::add(fo[ty * 32 + tx], vec_norm(sx * sx + sy * sy + sz * sz) * dt16);
        }
        px = hx; py = hy; pz = hz;
    }
    if (abort_flag) {
        if (tid == PRODUCER)
            for (int q = waited + 1; q < issued; ++q) mbar_wait_bounded(&bars[q % S], uint32_t((q / S) & 1));
    }
}

// Grid: (ceil(nx/32), ceil(ny/TY), ceil(nz/lz)) CTAs of 32 x TY threads.
template <typename real, int TY, int S>
__global__ void __launch_bounds__(32 * TY)
yee_hflu_tma(const StepArgs<real> a, const __grid_constant__ TmaMaps m, long long n, int lz, int* err)
{
    using T = HFluTile<real, TY>;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double tf[3];
    __shared__ int abort_flag;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    real* xs = reinterpret_cast<real*>(base + S * T::STAGE);
    Cpx<real>* uH = reinterpret_cast<Cpx<real>*>(xs + 2 * T::XS);
    uint64_t* bars = reinterpret_cast<uint64_t*>(uH + (lz + 2));
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY, kb = blockIdx.z * lz, ke = min(kb + lz, a.nz);
    bool gen, src;
    hflu_class<real, TY>(a, i0, j0, gen, src);
    if (gen) hflu_march<real, TY, S, true, true>(a, m, n, i0, j0, kb, ke, err, base, xs, uH, bars, tf, abort_flag);
    else if (src) hflu_march<real, TY, S, false, true>(a, m, n, i0, j0, kb, ke, err, base, xs, uH, bars, tf, abort_flag);
    else hflu_march<real, TY, S, false, false>(a, m, n, i0, j0, kb, ke, err, base, xs, uH, bars, tf, abort_flag);
}

}  // namespace fdtd
