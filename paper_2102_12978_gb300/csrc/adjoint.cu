// adjoint.cu -- reverse-time adjoint of the fused Yee step and the gradient
// of a loss on E with respect to the per-column antenna weights.
//
// The forward step (Section 4 leapfrog, CPML, PEC, soft source of Eq. 13) is
// linear in the state (E, H, CPML psi) plus a source term that is linear in
// the weighted coefficients B = w_amp e^{i w_phase} A.  Its exact discrete
// transpose, applied backwards in time, carries the adjoint state; the paper
// has no gradient computation, this is the transpose of the scheme above.
//
// One reverse step of forward step n (adjoints of E^{n+1}, H^{n+1/2}, psi in;
// of E^n, H^{n-1/2}, psi out), per z plane k, mirrors the forward's data flow:
//   * E side, tile plus a one-cell halo: e' = adjoint of E^{n+1} with the PEC
//     entries zeroed; per E cell the transposed-difference terms t (curl
//     coefficient x e' plus the CPML term a x psi-bar, psi-bar carried in a
//     ping-pong pair so halo readers see the old value);
//   * H side, tile plus the low halo: h' = h + gathered differences of t over
//     the forward neighbours (i+1, j+1, k+1), then the per-H-cell terms s;
//   * E side, own cells: e_new = e' + gathered differences of s over the
//     backward neighbours (i-1, j-1, k-1).
// The source gradient is g_c(col) = sum over steps and planes of
// lambda f e^{i (beta z_k - Phi_n)}, with lambda = e' (E points) or h'
// (H points); dL/dw follows per column as Re{e^{i phi} A g} and
// -w Im{e^{i phi} A g} summed over components.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "grid_impl.h"
#include "yee_tma.cuh"

namespace fdtd {

template <typename real>
struct AdjArgs {
    StepArgs<real> f;           // the forward grid's geometry, coefficients, antenna
    const real* ein[3];         // adjoint of E (read copy)
    real* eout[3];
    const real* hin[3];         // adjoint of H
    real* hout[3];
    const real* qx_in[2];       // adjoint of E-side psi, x shell (Eyx, Ezx)
    real* qx_out[2];
    const real* qy_in[2];       // y shell (Exy, Ezy)
    real* qy_out[2];
    const real* px_in[2];       // adjoint of H-side psi, x shell (Hyx, Hzx)
    real* px_out[2];
    const real* py_in[2];       // y shell (Hxy, Hzy)
    real* py_out[2];
    double2* grad;              // [6][ny][nx] sum of lambda f e^{i (beta z - Phi)}
};

template <typename real, int TY>
struct AdjTile {
    static constexpr int TX = 32, PX = TX + 2, PY = TY + 2, P = PX * PY, NT = TX * TY;
    // ring of E-side terms (3 planes x 9 values) and of H-side terms (2 x 6)
    static constexpr size_t smem_bytes(int lz) { return (27 + 12) * size_t(P) * sizeof(real) + 2 * size_t(lz + 3) * 2 * sizeof(real) + 64; }
};

// E-side terms of one cell at plane pw: t[0..5] = t_Ex_y, t_Ex_z, t_Ey_x,
// t_Ey_z, t_Ez_x, t_Ez_y; e[0..2] = e'.  Writes the carried psi adjoint of
// own cells (store).
template <typename real>
__device__ __forceinline__ void adj_eterms(const AdjArgs<real>& A, int i, int j, int pw, bool store, real t[6],
                                           real e[3])
{
    const StepArgs<real>& a = A.f;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    if (i < 0 || j < 0 || i >= nx || j >= ny) {
        for (int c = 0; c < 6; ++c) t[c] = real(0);
        e[0] = e[1] = e[2] = real(0);
        return;
    }
    const int g = pw * pitch * ny + j * pitch + i;
    real ex = A.ein[0][g], ey = A.ein[1][g], ez = A.ein[2][g];
    if (j == 0) { ex = real(0); ez = real(0); }   // PEC: E^{n+1} forced to zero there
    if (i == 0) { ey = real(0); ez = real(0); }
    e[0] = ex; e[1] = ey; e[2] = ez;
    const real cex = a.cex[i], cey = a.cey[j];
    t[0] = cey * ex;        // on dHz/dy in Ex
    t[1] = -a.cz * ex;      // on dHy/dz in Ex
    t[2] = -cex * ey;       // on dHz/dx in Ey
    t[3] = a.cz * ey;       // on dHx/dz in Ey
    t[4] = cex * ez;        // on dHy/dx in Ez
    t[5] = -cey * ez;       // on dHx/dy in Ez
    const int npml = a.npml, w2 = 2 * npml;
    if (npml > 0 && (i < npml || i >= nx - npml)) {
        const int ii = i < npml ? i : i - nx + w2;
        const int q = (pw * ny + j) * w2 + ii;
        const real b = a.bex[ii], aa = a.aex[ii];
        const real qyx = A.qx_in[0][q] - ey;      // Ey -= psi_Eyx
        const real qzx = A.qx_in[1][q] + ez;      // Ez += psi_Ezx
        t[2] += aa * qyx;
        t[4] += aa * qzx;
        if (store) { A.qx_out[0][q] = b * qyx; A.qx_out[1][q] = b * qzx; }
    }
    if (npml > 0 && (j < npml || j >= ny - npml)) {
        const int jj = j < npml ? j : j - ny + w2;
        const int q = (pw * w2 + jj) * pitch + i;
        const real b = a.bey[jj], aa = a.aey[jj];
        const real qxy = A.qy_in[0][q] + ex;      // Ex += psi_Exy
        const real qzy = A.qy_in[1][q] - ez;      // Ez -= psi_Ezy
        t[0] += aa * qxy;
        t[5] += aa * qzy;
        if (store) { A.qy_out[0][q] = b * qxy; A.qy_out[1][q] = b * qzy; }
    }
}

// H-side: h' from h and the E-side terms (t0: plane k, t1: plane k+1, ring
// index r of (i, j)); then s[0..5] = s_Hx_y, s_Hx_z, s_Hy_x, s_Hy_z, s_Hz_x, s_Hz_y.
template <typename real, int PX, int P>
__device__ __forceinline__ void adj_hterms(const AdjArgs<real>& A, int i, int j, int pw, bool store,
                                           const real* t0, const real* t1, int r, real hp[3], real s[6])
{
    const StepArgs<real>& a = A.f;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    const int g = pw * pitch * ny + j * pitch + i;
    real hx = A.hin[0][g], hy = A.hin[1][g], hz = A.hin[2][g];
    // t layout in the ring: value c of cell r at t[c * P + r]
    hx += (t0[3 * P + r] - t1[3 * P + r]) + (t0[5 * P + r] - t0[5 * P + r + PX]);
    hy += (t0[1 * P + r] - t1[1 * P + r]) + (t0[4 * P + r] - t0[4 * P + r + 1]);
    hz += (t0[0 * P + r] - t0[0 * P + r + PX]) + (t0[2 * P + r] - t0[2 * P + r + 1]);
    hp[0] = hx; hp[1] = hy; hp[2] = hz;
    const real chx = a.chx[i], chy = a.chy[j];
    s[0] = -chy * hx;      // on dEz/dy in Hx
    s[1] = a.cz * hx;      // on dEy/dz in Hx
    s[2] = chx * hy;       // on dEz/dx in Hy
    s[3] = -a.cz * hy;     // on dEx/dz in Hy
    s[4] = -chx * hz;      // on dEy/dx in Hz
    s[5] = chy * hz;       // on dEx/dy in Hz
    const int npml = a.npml, w2 = 2 * npml;
    if (npml > 0 && (i < npml || i >= nx - npml)) {
        const int ii = i < npml ? i : i - nx + w2;
        const int q = (pw * ny + j) * w2 + ii;
        const real b = a.bhx[ii], aa = a.ahx[ii];
        const real pyx = A.px_in[0][q] + hy;      // Hy += psi_Hyx
        const real pzx = A.px_in[1][q] - hz;      // Hz -= psi_Hzx
        s[2] += aa * pyx;
        s[4] += aa * pzx;
        if (store) { A.px_out[0][q] = b * pyx; A.px_out[1][q] = b * pzx; }
    }
    if (npml > 0 && (j < npml || j >= ny - npml)) {
        const int jj = j < npml ? j : j - ny + w2;
        const int q = (pw * w2 + jj) * pitch + i;
        const real b = a.bhy[jj], aa = a.ahy[jj];
        const real pxy = A.py_in[0][q] - hx;      // Hx -= psi_Hxy
        const real pzy = A.py_in[1][q] + hz;      // Hz += psi_Hzy
        s[0] += aa * pxy;
        s[5] += aa * pzy;
        if (store) { A.py_out[0][q] = b * pxy; A.py_out[1][q] = b * pzy; }
    }
}

template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_adjoint_step(const AdjArgs<real> A, long long n, int lz)
{
    using T = AdjTile<real, TY>;
    constexpr int TX = T::TX, PX = T::PX, P = T::P, NT = T::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* tr = reinterpret_cast<real*>(smem_raw);   // [3][9][P]: t (6) and e' (3)
    real* sr = tr + 27 * P;                          // [2][6][P]
    Cpx<real>* uE = reinterpret_cast<Cpx<real>*>(sr + 12 * P);
    Cpx<real>* uH = uE + (lz + 3);
    __shared__ double tf[6];

    const StepArgs<real>& a = A.f;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int kb = blockIdx.z * lz;
    const int ke = min(kb + lz, a.nz);
    const int nx = a.nx, ny = a.ny, nz = a.nz, pitch = a.pitch;
    const int i = i0 + tx, j = j0 + ty;
    const bool own = i < nx && j < ny;
    const int so = (ty + 1) * PX + (tx + 1);

    if (tid == 0) {
        double c, s, f;
        source_time(a.st, (double(n) + 0.5) * a.dt, c, s, f);
        tf[3] = c; tf[4] = s; tf[5] = f;
        source_time(a.st, (double(n) + 1.0) * a.dt, c, s, f);
        tf[0] = c; tf[1] = s; tf[2] = f;
    }
    for (int q = tid; q < 39 * P; q += NT) tr[q] = real(0);
    __syncthreads();
    const int Q = ke - kb + 3;
    if (a.smask) {
        for (int q = tid; q < Q; q += NT) {
            const int p = kb - 1 + q;
            const int pw = p < 0 ? p + nz : (p >= nz ? p - nz : p);
            const double2 z = a.zph[pw];
            uE[q].x = real((z.x * tf[0] + z.y * tf[1]) * tf[2]);
            uE[q].y = real((z.y * tf[0] - z.x * tf[1]) * tf[2]);
            uH[q].x = real((z.x * tf[3] + z.y * tf[4]) * tf[5]);
            uH[q].y = real((z.y * tf[3] - z.x * tf[4]) * tf[5]);
        }
    }
    const uint8_t mk = (own && a.smask) ? a.smask[j * nx + i] : uint8_t(0);
    Cpx<real> gacc[6];
    for (int c = 0; c < 6; ++c) { gacc[c].x = real(0); gacc[c].y = real(0); }

    // E-side terms of plane p into ring slot (p + 3) % 3 (three slots: plane
    // k+1 is filled while the previous iteration may still read plane k-1);
    // the region's cells are shared out flatly over the CTA
    auto tslot = [&](int p) { return tr + ((p + 3) % 3) * 9 * P; };
    auto fill_t = [&](int p) {
        const int pw = ((p % nz) + nz) % nz;
        real* dst = tslot(p);
        const bool own_plane = p >= kb && p < ke;
        for (int r = tid; r < P; r += NT) {
            const int ri = r % PX, rj = r / PX;
            const int ci = i0 - 1 + ri, cj = j0 - 1 + rj;
            const bool owner = own_plane && ri >= 1 && ri <= TX && rj >= 1 && rj <= TY;
            real t[6], e[3];
            adj_eterms<real>(A, ci, cj, pw, owner, t, e);
            for (int c = 0; c < 6; ++c) dst[c * P + r] = t[c];
            for (int c = 0; c < 3; ++c) dst[(6 + c) * P + r] = e[c];
        }
    };

    // H cells of this thread: own, plus one of the low-halo cells
    int hi = -1, hj = -1, hs = 0;
    if (tid < TX) { hi = i0 + tid; hj = j0 - 1; hs = tid + 1; }
    else if (tid < TX + TY + 1) { hi = i0 - 1; hj = j0 - 1 + (tid - TX); hs = (tid - TX) * PX; }
    const bool halo_in = hi >= 0 && hj >= 0 && hi < nx && hj < ny;

    fill_t(kb - 1);
    #pragma unroll 1
    for (int k = kb - 1; k < ke; ++k) {
        const int q = k - kb + 1;
        fill_t(k + 1);
        __syncthreads();   // t of planes k, k+1 ready; readers of plane k-2's s slot done
        const int kw = ((k % nz) + nz) % nz;
        const bool write_k = k >= kb;
        const real* t0 = tslot(k);
        const real* t1 = tslot(k + 1);
        real* sk = sr + (k & 1) * 6 * P;
        if (own) {
            real hp[3], s[6];
            adj_hterms<real, PX, P>(A, i, j, kw, write_k, t0, t1, so, hp, s);
            for (int c = 0; c < 6; ++c) sk[c * P + so] = s[c];
            if (write_k) {
                const int g = kw * pitch * ny + j * pitch + i;
                A.hout[0][g] = hp[0]; A.hout[1][g] = hp[1]; A.hout[2][g] = hp[2];
                if (mk & 0x38) {
                    const Cpx<real> u = uH[q];
                    for (int c = 3; c < 6; ++c)
                        if (mk & (1 << c)) { gacc[c].x += hp[c - 3] * u.x; gacc[c].y += hp[c - 3] * u.y; }
                }
            }
        } else {
            for (int c = 0; c < 6; ++c) sk[c * P + so] = real(0);
        }
        if (tid < TX + TY + 1) {
            if (halo_in) {
                real hp[3], s[6];
                adj_hterms<real, PX, P>(A, hi, hj, kw, false, t0, t1, hs, hp, s);
                for (int c = 0; c < 6; ++c) sk[c * P + hs] = s[c];
            } else {
                for (int c = 0; c < 6; ++c) sk[c * P + hs] = real(0);
            }
        }
        __syncthreads();   // s of planes k, k-1 ready
        if (write_k && own) {
            const real* s0 = sr + (k & 1) * 6 * P;
            const real* s1 = sr + ((k - 1) & 1) * 6 * P;
            const real ex = t0[6 * P + so], ey = t0[7 * P + so], ez = t0[8 * P + so];
            // backward differences of s (i-1, j-1, k-1)
            const real nex = ex + (s1[3 * P + so] - s0[3 * P + so]) + (s0[5 * P + so - PX] - s0[5 * P + so]);
            const real ney = ey + (s1[1 * P + so] - s0[1 * P + so]) + (s0[4 * P + so - 1] - s0[4 * P + so]);
            const real nez = ez + (s0[0 * P + so - PX] - s0[0 * P + so]) + (s0[2 * P + so - 1] - s0[2 * P + so]);
            const int g = kw * pitch * ny + j * pitch + i;
            A.eout[0][g] = nex; A.eout[1][g] = ney; A.eout[2][g] = nez;
            if (mk & 0x07) {
                const Cpx<real> u = uE[q];
                const real ev[3] = {ex, ey, ez};
                for (int c = 0; c < 3; ++c)
                    if (mk & (1 << c)) { gacc[c].x += ev[c] * u.x; gacc[c].y += ev[c] * u.y; }
            }
        }
    }
    if (mk) {
        const int ncol = nx * ny, col = j * nx + i;
        for (int c = 0; c < 6; ++c)
            if (mk & (1 << c)) {
                atomicAdd(&A.grad[c * ncol + col].x, double(gacc[c].x));
                atomicAdd(&A.grad[c * ncol + col].y, double(gacc[c].y));
            }
    }
}

// dL/dw per column from the accumulated g: sum over components of
// Re{e^{i phi} A g} (amplitude) and -w Im{e^{i phi} A g} (phase).
__global__ void adjoint_weight_grad(const double2* __restrict__ grad, const double2* __restrict__ coef_unw,
                                    const double* __restrict__ w_amp, const double* __restrict__ w_phase, int ncol,
                                    double* __restrict__ d_amp, double* __restrict__ d_phase)
{
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < ncol; col += gridDim.x * blockDim.x) {
        double sa = 0.0, sp = 0.0;
        double s, c;
        sincos(w_phase[col], &s, &c);
        for (int comp = 0; comp < 6; ++comp) {
            const double2 A = coef_unw[comp * ncol + col], g = grad[comp * ncol + col];
            const double zr = c * A.x - s * A.y, zi = c * A.y + s * A.x;   // e^{i phi} A
            const double pr = zr * g.x - zi * g.y, pi = zr * g.y + zi * g.x;
            sa += pr;
            sp += -w_amp[col] * pi;
        }
        d_amp[col] = sa;
        d_phase[col] = sp;
    }
}

template <typename real>
__global__ void probe_gather(const real* __restrict__ f, const int* __restrict__ cells, long long n,
                             real* __restrict__ out)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        out[p] = f[cells[p]];
}

template <typename real>
__global__ void probe_inject(real* __restrict__ f, const int* __restrict__ cells, long long n,
                             const real* __restrict__ v)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x)
        f[cells[p]] += v[p];
}

}  // namespace fdtd

using namespace fdtd;

struct fdtd_adjoint {
    fdtd_grid* g;
    int component;
    int64_t nprobes;
    void* arena;
    size_t bytes;
    int64_t n;               // the adjoint sits at forward step n
    int cur;
    // arena offsets
    size_t e[2][3], h[2][3], qx[2][2], qy[2][2], px[2][2], py[2][2];
    size_t grad, cells, dyn_bytes, wout;
    int lz;
};

namespace {

static size_t al256(size_t v) { return (v + 255) / 256 * 256; }

static void adj_layout(const fdtd_grid* g, int64_t nprobes, fdtd_adjoint* a, size_t* total)
{
    const Layout& L = g->L;
    const size_t b = L.elem;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = al256(off + bytes); return o; };
    for (int buf = 0; buf < 2; ++buf) {
        for (int c = 0; c < 3; ++c) { a->e[buf][c] = take(L.field_elems * b); a->h[buf][c] = take(L.field_elems * b); }
        for (int c = 0; c < 2; ++c) {
            a->qx[buf][c] = take(L.psx_elems * b); a->qy[buf][c] = take(L.psy_elems * b);
            a->px[buf][c] = take(L.psx_elems * b); a->py[buf][c] = take(L.psy_elems * b);
        }
    }
    a->grad = take(6 * size_t(g->desc.nx) * g->desc.ny * 16);
    a->dyn_bytes = off;
    a->wout = take(2 * size_t(g->desc.nx) * g->desc.ny * 8);
    a->cells = take(size_t(nprobes > 0 ? nprobes : 1) * 4);
    *total = off;
}

template <typename real>
AdjArgs<real> adj_args(const fdtd_adjoint* ad)
{
    AdjArgs<real> A;
    A.f = make_args<real>(ad->g, ad->g->cur);
    char* M = static_cast<char*>(ad->arena);
    const int c0 = ad->cur, c1 = ad->cur ^ 1;
    for (int c = 0; c < 3; ++c) {
        A.ein[c] = reinterpret_cast<const real*>(M + ad->e[c0][c]);
        A.eout[c] = reinterpret_cast<real*>(M + ad->e[c1][c]);
        A.hin[c] = reinterpret_cast<const real*>(M + ad->h[c0][c]);
        A.hout[c] = reinterpret_cast<real*>(M + ad->h[c1][c]);
    }
    for (int c = 0; c < 2; ++c) {
        A.qx_in[c] = reinterpret_cast<const real*>(M + ad->qx[c0][c]);
        A.qx_out[c] = reinterpret_cast<real*>(M + ad->qx[c1][c]);
        A.qy_in[c] = reinterpret_cast<const real*>(M + ad->qy[c0][c]);
        A.qy_out[c] = reinterpret_cast<real*>(M + ad->qy[c1][c]);
        A.px_in[c] = reinterpret_cast<const real*>(M + ad->px[c0][c]);
        A.px_out[c] = reinterpret_cast<real*>(M + ad->px[c1][c]);
        A.py_in[c] = reinterpret_cast<const real*>(M + ad->py[c0][c]);
        A.py_out[c] = reinterpret_cast<real*>(M + ad->py[c1][c]);
    }
    A.grad = reinterpret_cast<double2*>(M + ad->grad);
    return A;
}

template <typename real, int TY>
cudaError_t adj_launch(fdtd_adjoint* ad, long long n)
{
    using T = AdjTile<real, TY>;
    const int lz = ad->lz;
    const size_t smem = T::smem_bytes(lz);
    static size_t attr = 0;
    if (smem > attr) {
        cudaError_t e = cudaFuncSetAttribute(yee_adjoint_step<real, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        attr = smem;
    }
    const fdtd_grid_desc& d = ad->g->desc;
    dim3 grid((d.nx + 31) / 32, (d.ny + TY - 1) / TY, (d.nz + lz - 1) / lz);
    yee_adjoint_step<real, TY><<<grid, dim3(32, TY), smem, ad->g->stream>>>(adj_args<real>(ad), n, lz);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gather(fdtd_adjoint* ad, void* out)
{
    const fdtd_grid* g = ad->g;
    const char* A = static_cast<const char*>(g->arena);
    const real* f = reinterpret_cast<const real*>(A + g->L.field[g->cur][ad->component]);
    const int* cells = reinterpret_cast<const int*>(static_cast<char*>(ad->arena) + ad->cells);
    int blocks = int((ad->nprobes + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    probe_gather<real><<<blocks, 256, 0, g->stream>>>(f, cells, ad->nprobes, static_cast<real*>(out));
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_inject(fdtd_adjoint* ad, const void* v)
{
    real* f = reinterpret_cast<real*>(static_cast<char*>(ad->arena) + ad->e[ad->cur][ad->component]);
    const int* cells = reinterpret_cast<const int*>(static_cast<char*>(ad->arena) + ad->cells);
    int blocks = int((ad->nprobes + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    probe_inject<real><<<blocks, 256, 0, ad->g->stream>>>(f, cells, ad->nprobes, static_cast<const real*>(v));
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t fdtd_adjoint_required_bytes(const fdtd_grid* g, int64_t n_probes)
{
    if (!g || n_probes < 0) return 0;
    fdtd_adjoint tmp;
    size_t total = 0;
    adj_layout(g, n_probes, &tmp, &total);
    return total;
}

fdtd_status fdtd_adjoint_create(fdtd_grid* g, int component, const int64_t* probe_cells, int64_t n_probes,
                                void* arena, size_t bytes, fdtd_adjoint** out)
{
    if (!out) return fail(FDTD_EINVAL, "null output pointer");
    *out = nullptr;
    if (!g || !arena || component < 0 || component > 2 || n_probes < 0 || (n_probes > 0 && !probe_cells))
        return fail(FDTD_EINVAL, "invalid adjoint arguments");
    if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) return fail(FDTD_EINVAL, "arena not 256-byte aligned");
    if (!g->has_source) return fail(FDTD_ESTATE, "set the antenna source before creating its adjoint");
    fdtd_adjoint* a = new (std::nothrow) fdtd_adjoint();
    if (!a) return fail(FDTD_ENOMEM, "host allocation failed");
    size_t total = 0;
    adj_layout(g, n_probes, a, &total);
    if (bytes < total) { delete a; return fail(FDTD_ENOMEM, "adjoint arena of %zu bytes, %zu needed", bytes, total); }
    a->g = g;
    a->component = component;
    a->nprobes = n_probes;
    a->arena = arena;
    a->bytes = bytes;
    a->n = g->step;
    a->cur = 0;
    a->lz = g->desc.nz < 32 ? g->desc.nz : 32;
    // probe cells -> pitched element offsets
    const fdtd_grid_desc& d = g->desc;
    std::vector<int> off(size_t(n_probes > 0 ? n_probes : 1), 0);
    for (int64_t p = 0; p < n_probes; ++p) {
        const int64_t c = probe_cells[p];
        if (c < 0 || c >= int64_t(d.nx) * d.ny * d.nz) { delete a; return fail(FDTD_EINVAL, "probe cell %lld out of range", (long long)c); }
        const int64_t i = c % d.nx, r = c / d.nx, j = r % d.ny, k = r / d.ny;
        off[size_t(p)] = int((k * d.ny + j) * g->L.pitch + i);
    }
    fdtd_status st = cuda_check(cudaMemsetAsync(arena, 0, a->dyn_bytes, g->stream), "zero adjoint");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(static_cast<char*>(arena) + a->cells, off.data(), off.size() * 4,
                                        cudaMemcpyHostToDevice, g->stream), "upload probes");
    if (st == FDTD_OK) st = cuda_check(cudaStreamSynchronize(g->stream), "adjoint create");
    if (st != FDTD_OK) { delete a; return st; }
    *out = a;
    return FDTD_OK;
}

fdtd_status fdtd_adjoint_reset(fdtd_adjoint* a, int64_t n_end)
{
    if (!a || n_end < 0) return fail(FDTD_EINVAL, "invalid argument");
    a->n = n_end;
    a->cur = 0;
    return cuda_check(cudaMemsetAsync(a->arena, 0, a->dyn_bytes, a->g->stream), "reset adjoint");
}

fdtd_status fdtd_probe_read(fdtd_adjoint* a, void* dev_out)
{
    if (!a || !dev_out) return fail(FDTD_EINVAL, "null argument");
    if (a->nprobes == 0) return FDTD_OK;
    cudaError_t e = a->g->desc.precision == FDTD_F64 ? launch_gather<double>(a, dev_out) : launch_gather<float>(a, dev_out);
    return cuda_check(e, "probe gather");
}

fdtd_status fdtd_adjoint_step(fdtd_adjoint* a, int nsteps, const void* dLdE, int64_t ld)
{
    if (!a || nsteps < 0) return fail(FDTD_EINVAL, "invalid argument");
    if (nsteps > a->n) return fail(FDTD_EINVAL, "cannot step the adjoint before forward step 0");
    const size_t eb = a->g->L.elem;
    for (int s = 0; s < nsteps; ++s) {
        if (dLdE && a->nprobes > 0) {
            const void* row = static_cast<const char*>(dLdE) + size_t(s) * size_t(ld) * eb;
            cudaError_t e = eb == 8 ? launch_inject<double>(a, row) : launch_inject<float>(a, row);
            if (e != cudaSuccess) return cuda_check(e, "adjoint inject");
        }
        const long long n = a->n - 1;   // reverse forward step n
        cudaError_t e = eb == 8 ? adj_launch<double, 4>(a, n) : adj_launch<float, 8>(a, n);
        if (e != cudaSuccess) return cuda_check(e, "adjoint step");
        a->cur ^= 1;
        a->n -= 1;
    }
    return FDTD_OK;
}

int64_t fdtd_adjoint_position(const fdtd_adjoint* a) { return a ? a->n : -1; }

fdtd_status fdtd_adjoint_get(fdtd_adjoint* a, int component, void* dst)
{
    if (!a || !dst || component < 0 || component > 5) return fail(FDTD_EINVAL, "invalid argument");
    const fdtd_grid_desc& d = a->g->desc;
    const size_t b = a->g->L.elem;
    const size_t off = component < 3 ? a->e[a->cur][component] : a->h[a->cur][component - 3];
    fdtd_status st = cuda_check(cudaMemcpy2DAsync(dst, size_t(d.nx) * b, static_cast<char*>(a->arena) + off,
                                                  size_t(a->g->L.pitch) * b, size_t(d.nx) * b, size_t(d.ny) * d.nz,
                                                  cudaMemcpyDeviceToDevice, a->g->stream),
                                "copy adjoint field");
    if (st != FDTD_OK) return st;
    return fdtd_sync(a->g);
}

fdtd_status fdtd_adjoint_gradient(fdtd_adjoint* a, double* dLdw_amp, double* dLdw_phase, int on_device)
{
    if (!a || !dLdw_amp || !dLdw_phase) return fail(FDTD_EINVAL, "null argument");
    fdtd_grid* g = a->g;
    const int ncol = g->desc.nx * g->desc.ny;
    char* G = static_cast<char*>(g->arena);
    char* M = static_cast<char*>(a->arena);
    double* out = reinterpret_cast<double*>(M + a->wout);
    adjoint_weight_grad<<<4 * (g->sm_count > 0 ? g->sm_count : 152), 256, 0, g->stream>>>(
        reinterpret_cast<const double2*>(M + a->grad), reinterpret_cast<const double2*>(G + g->L.scoef_unw),
        reinterpret_cast<const double*>(G + g->L.wamp), reinterpret_cast<const double*>(G + g->L.wphase), ncol, out,
        out + ncol);
    fdtd_status st = cuda_check(cudaGetLastError(), "weight gradient");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (st == FDTD_OK) st = cuda_check(cudaMemcpyAsync(dLdw_amp, out, size_t(ncol) * 8, kind, g->stream), "copy gradient");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(dLdw_phase, out + ncol, size_t(ncol) * 8, kind, g->stream), "copy gradient");
    if (st != FDTD_OK) return st;
    return fdtd_sync(g);
}

void fdtd_adjoint_destroy(fdtd_adjoint* a) { delete a; }

}  // extern "C"
