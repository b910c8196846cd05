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
// of E^n, H^{n-1/2}, psi out) mirrors the forward's data flow:
//   * e' = adjoint of E^{n+1} with the PEC entries zeroed; per E cell the
//     transposed-difference terms t (curl coefficient x e' plus the CPML term
//     a x psi-bar, psi-bar carried in a ping-pong pair so that neighbours
//     read the old value);
//   * h' = h + gathered differences of t over the forward neighbours
//     (i+1, j+1, k+1), then the per-H-cell terms s;
//   * e_new = e' + gathered differences of s over the backward neighbours
//     (i-1, j-1, k-1).
// It runs as two cell-parallel passes (h', then e_new) and a small kernel
// over the antenna columns for the source gradient
// g_c(col) = sum over steps and planes of lambda f e^{i (beta z_k - Phi_n)},
// with lambda = e' (E points) or h' (H points); dL/dw follows per column as
// Re{e^{i phi} A g} and -w Im{e^{i phi} A g} summed over components.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "grid_impl.h"
#include "yee_cell.cuh"
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

// ---- cell-parallel reverse step: two passes and a source-gradient kernel.
//
// Pass A (adj_h_cell): h' = lambda_H + gathered differences of the E-side
// terms t over the forward neighbours (i+1, j+1, k+1); the own cell's t also
// carries the E-side psi adjoint (written to the other copy).
// Pass B (adj_e_cell): e_new = e' + gathered differences of the H-side terms
// s over the backward neighbours (i-1, j-1, k-1), s from h' of pass A; the
// own cell's s carries the H-side psi adjoint.
// Every t and s a cell needs is recomputed from the read copies (neighbours
// never write what a cell reads), so both passes are one thread per cell with
// no shared memory or barrier, like the forward cell passes.

// E-side terms t[0..5] of (i, j, pw) and e' (PEC-zeroed adjoint of E^{n+1});
// zero outside the grid.  GEN: the cell may be outside the grid or in the
// shell.
template <typename real, bool GEN>
__device__ __forceinline__ void adj_t(const AdjArgs<real>& A, int i, int j, int pw, bool store, real t[6], real e[3])
{
    const StepArgs<real>& a = A.f;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    if (GEN && (i < 0 || j < 0 || i >= nx || j >= ny)) {
        for (int c = 0; c < 6; ++c) t[c] = real(0);
        e[0] = e[1] = e[2] = real(0);
        return;
    }
    const int g = pw * pitch * ny + j * pitch + i;
    real ex = fld<true>(A.ein[0] + g), ey = fld<true>(A.ein[1] + g), ez = fld<true>(A.ein[2] + g);
    if (GEN) {
        if (j == 0) { ex = real(0); ez = real(0); }   // PEC: E^{n+1} forced to zero there
        if (i == 0) { ey = real(0); ez = real(0); }
    }
    e[0] = ex; e[1] = ey; e[2] = ez;
    const real cex = __ldg(a.cex + i), cey = __ldg(a.cey + j);
    t[0] = cey * ex;        // on dHz/dy in Ex
    t[1] = -a.cz * ex;      // on dHy/dz in Ex
    t[2] = -cex * ey;       // on dHz/dx in Ey
    t[3] = a.cz * ey;       // on dHx/dz in Ey
    t[4] = cex * ez;        // on dHy/dx in Ez
    t[5] = -cey * ez;       // on dHx/dy in Ez
    if (GEN && a.npml > 0) {
        const int npml = a.npml, w2 = 2 * npml;
        if (i < npml || i >= nx - npml) {
            const int ii = i < npml ? i : i - nx + w2;
            const int q = (pw * ny + j) * w2 + ii;
            const real b = a.bex[ii], aa = a.aex[ii];
            const real qyx = A.qx_in[0][q] - ey;      // Ey -= psi_Eyx
            const real qzx = A.qx_in[1][q] + ez;      // Ez += psi_Ezx
            t[2] += aa * qyx;
            t[4] += aa * qzx;
            if (store) { A.qx_out[0][q] = b * qyx; A.qx_out[1][q] = b * qzx; }
        }
        if (j < npml || j >= ny - npml) {
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
}

// H-side terms s[0..5] of (i, j, pw) from h' (pass A's output, A.hout);
// zero outside the grid.
template <typename real, bool GEN>
__device__ __forceinline__ void adj_s(const AdjArgs<real>& A, int i, int j, int pw, bool store, real s[6])
{
    const StepArgs<real>& a = A.f;
    const int nx = a.nx, ny = a.ny, pitch = a.pitch;
    if (GEN && (i < 0 || j < 0 || i >= nx || j >= ny)) {
        for (int c = 0; c < 6; ++c) s[c] = real(0);
        return;
    }
    const int g = pw * pitch * ny + j * pitch + i;
    const real hx = fld<true>(A.hout[0] + g), hy = fld<true>(A.hout[1] + g), hz = fld<true>(A.hout[2] + g);
    const real chx = __ldg(a.chx + i), chy = __ldg(a.chy + j);
    s[0] = -chy * hx;      // on dEz/dy in Hx
    s[1] = a.cz * hx;      // on dEy/dz in Hx
    s[2] = chx * hy;       // on dEz/dx in Hy
    s[3] = -a.cz * hy;     // on dEx/dz in Hy
    s[4] = -chx * hz;      // on dEy/dx in Hz
    s[5] = chy * hz;       // on dEx/dy in Hz
    if (GEN && a.npml > 0) {
        const int npml = a.npml, w2 = 2 * npml;
        if (i < npml || i >= nx - npml) {
            const int ii = i < npml ? i : i - nx + w2;
            const int q = (pw * ny + j) * w2 + ii;
            const real b = a.bhx[ii], aa = a.ahx[ii];
            const real pyx = A.px_in[0][q] + hy;      // Hy += psi_Hyx
            const real pzx = A.px_in[1][q] - hz;      // Hz -= psi_Hzx
            s[2] += aa * pyx;
            s[4] += aa * pzx;
            if (store) { A.px_out[0][q] = b * pyx; A.px_out[1][q] = b * pzx; }
        }
        if (j < npml || j >= ny - npml) {
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
}

template <typename real, bool GEN>
__device__ __forceinline__ void adj_h_cell(const AdjArgs<real>& A, int i, int j, int k)
{
    const StepArgs<real>& a = A.f;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    if (GEN && (i >= nx || j >= ny)) return;
    const int kp = k + 1 == nz ? 0 : k + 1;
    real t[6], e[3], tx[6], ty[6], tz[6];
    adj_t<real, GEN>(A, i, j, k, true, t, e);
    adj_t<real, GEN>(A, i + 1, j, k, false, tx, e);
    adj_t<real, GEN>(A, i, j + 1, k, false, ty, e);
    adj_t<real, GEN>(A, i, j, kp, false, tz, e);
    const int g = k * a.pitch * ny + j * a.pitch + i;
    real hx = fld<true>(A.hin[0] + g), hy = fld<true>(A.hin[1] + g), hz = fld<true>(A.hin[2] + g);
    hx += (t[3] - tz[3]) + (t[5] - ty[5]);
    hy += (t[1] - tz[1]) + (t[4] - tx[4]);
    hz += (t[0] - ty[0]) + (t[2] - tx[2]);
    A.hout[0][g] = hx; A.hout[1][g] = hy; A.hout[2][g] = hz;
}

template <typename real, bool GEN>
__device__ __forceinline__ void adj_e_cell(const AdjArgs<real>& A, int i, int j, int k)
{
    const StepArgs<real>& a = A.f;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    if (GEN && (i >= nx || j >= ny)) return;
    const int km = k == 0 ? nz - 1 : k - 1;
    real s[6], sx[6], sy[6], sz[6];
    adj_s<real, GEN>(A, i, j, k, true, s);
    adj_s<real, GEN>(A, i - 1, j, k, false, sx);
    adj_s<real, GEN>(A, i, j - 1, k, false, sy);
    adj_s<real, GEN>(A, i, j, km, false, sz);
    const int g = k * a.pitch * ny + j * a.pitch + i;
    real ex = fld<true>(A.ein[0] + g), ey = fld<true>(A.ein[1] + g), ez = fld<true>(A.ein[2] + g);
    if (GEN) {
        if (j == 0) { ex = real(0); ez = real(0); }
        if (i == 0) { ey = real(0); ez = real(0); }
    }
    A.eout[0][g] = ex + (sz[3] - s[3]) + (sy[5] - s[5]);
    A.eout[1][g] = ey + (sz[1] - s[1]) + (sx[4] - s[4]);
    A.eout[2][g] = ez + (sy[0] - s[0]) + (sx[2] - s[2]);
}

// Grid: (ceil(nx/32), ceil(ny/TY), nz) CTAs of 32 x TY threads, one cell each.
// GEN blocks: cells or the neighbours they read reach a wall, a ragged edge
// or the shell.
template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_adj_h_cell(const AdjArgs<real> A)
{
    const StepArgs<real>& a = A.f;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY, k = blockIdx.z;
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    const bool gen = i0 == 0 || j0 == 0 || i0 + 32 >= nx || j0 + TY >= ny ||
                     (npml > 0 && (i0 < npml || i0 + 32 >= nx - npml || j0 < npml || j0 + TY >= ny - npml));
    if (gen) adj_h_cell<real, true>(A, i0 + threadIdx.x, j0 + threadIdx.y, k);
    else adj_h_cell<real, false>(A, i0 + threadIdx.x, j0 + threadIdx.y, k);
}

template <typename real, int TY>
__global__ void __launch_bounds__(32 * TY)
yee_adj_e_cell(const AdjArgs<real> A)
{
    const StepArgs<real>& a = A.f;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TY, k = blockIdx.z;
    const int nx = a.nx, ny = a.ny, npml = a.npml;
    const bool gen = i0 == 0 || j0 == 0 || i0 + 32 >= nx || j0 + TY >= ny ||
                     (npml > 0 && (i0 - 1 < npml || i0 + 31 >= nx - npml || j0 - 1 < npml || j0 + TY - 1 >= ny - npml));
    if (gen) adj_e_cell<real, true>(A, i0 + threadIdx.x, j0 + threadIdx.y, k);
    else adj_e_cell<real, false>(A, i0 + threadIdx.x, j0 + threadIdx.y, k);
}

// Source gradient of one reverse step: for each antenna column (one warp per
// column; lanes share out the planes) and component c with an antenna point,
// g_c(col) += sum_k lambda_c(k) Re/Im{u_c(k)}, lambda = h' (H points, pass
// A's output) or e' (E points: the PEC-zeroed adjoint of E^{n+1}), u_c(k) =
// f e^{i (beta z_k - Phi)} at the component's time, in FP64.
template <typename real>
__global__ void adj_source_grad(const AdjArgs<real> A, const int* __restrict__ cols, int ncols, double2 te,
                                double2 th)
{
    const StepArgs<real>& a = A.f;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int nx = a.nx, ny = a.ny, nz = a.nz, plane = a.pitch * ny;
    for (int w = warp; w < ncols; w += nwarps) {
        const int col = cols[w];
        const int j = col / nx, i = col - j * nx;
        const uint8_t mk = a.smask[col];
        double2 acc[6];
        for (int c = 0; c < 6; ++c) acc[c] = make_double2(0.0, 0.0);
        for (int k = lane; k < nz; k += 32) {
            const double2 z = a.zph[k];
            const double2 ue = make_double2(z.x * te.x - z.y * te.y, z.x * te.y + z.y * te.x);
            const double2 uh = make_double2(z.x * th.x - z.y * th.y, z.x * th.y + z.y * th.x);
            const int g = k * plane + j * a.pitch + i;
            for (int c = 0; c < 3; ++c)
                if (mk & (1 << c)) {
                    real v = A.ein[c][g];
                    if ((j == 0 && c != 1) || (i == 0 && c != 0)) v = real(0);   // PEC
                    acc[c].x += double(v) * ue.x;
                    acc[c].y += double(v) * ue.y;
                }
            for (int c = 3; c < 6; ++c)
                if (mk & (1 << c)) {
                    const double v = double(A.hout[c - 3][g]);
                    acc[c].x += v * uh.x;
                    acc[c].y += v * uh.y;
                }
        }
        for (int c = 0; c < 6; ++c) {
            if (!(mk & (1 << c))) continue;
            double x = acc[c].x, y = acc[c].y;
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_down_sync(0xffffffffu, x, o);
                y += __shfl_down_sync(0xffffffffu, y, o);
            }
            if (lane == 0) {
                double2& gr = A.grad[c * nx * ny + col];
                gr.x += x;
                gr.y += y;
            }
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
    size_t grad, cells, dyn_bytes, wout, acols;
    int nacols;              // antenna columns (any component)
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
    a->acols = take(size_t(g->desc.nx) * g->desc.ny * 4);
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

// One reverse step of forward step n: the two cell passes and the source
// gradient (time factors of step n evaluated on the host in FP64).
template <typename real, int TY>
cudaError_t adj_cell_launch(fdtd_adjoint* ad, long long n)
{
    const fdtd_grid* g = ad->g;
    const fdtd_grid_desc& d = g->desc;
    const AdjArgs<real> A = adj_args<real>(ad);
    const dim3 grid((d.nx + 31) / 32, (d.ny + TY - 1) / TY, d.nz), block(32, TY);
    yee_adj_h_cell<real, TY><<<grid, block, 0, g->stream>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    yee_adj_e_cell<real, TY><<<grid, block, 0, g->stream>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess || ad->nacols == 0) return e;
    double c, sn, f;
    source_time(g->srct, (double(n) + 1.0) * g->dt, c, sn, f);
    const double2 te = make_double2(f * c, -f * sn);
    source_time(g->srct, (double(n) + 0.5) * g->dt, c, sn, f);
    const double2 th = make_double2(f * c, -f * sn);
    const int* cols = reinterpret_cast<const int*>(static_cast<char*>(ad->arena) + ad->acols);
    const int threads = 256, blocks = (ad->nacols * 32 + threads - 1) / threads;
    adj_source_grad<real><<<blocks < 4096 ? blocks : 4096, threads, 0, g->stream>>>(A, cols, ad->nacols, te, th);
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
    if (needs_cell_passes(g)) return fail(FDTD_EINVAL, "no adjoint for grids with z walls or a wall source");
    if (!g->has_source) return fail(FDTD_ESTATE, "set the antenna source before creating its adjoint");
    const fdtd_status dev_st = check_device(g, "fdtd_adjoint_create");
    if (dev_st != FDTD_OK) return dev_st;
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
    // probe cells -> pitched element offsets
    const fdtd_grid_desc& d = g->desc;
    std::vector<int> off(size_t(n_probes > 0 ? n_probes : 1), 0);
    for (int64_t p = 0; p < n_probes; ++p) {
        const int64_t c = probe_cells[p];
        if (c < 0 || c >= int64_t(d.nx) * d.ny * d.nz) { delete a; return fail(FDTD_EINVAL, "probe cell %lld out of range", (long long)c); }
        const int64_t i = c % d.nx, r = c / d.nx, j = r % d.ny, k = r / d.ny;
        off[size_t(p)] = int((k * d.ny + j) * g->L.pitch + i);
    }
    // antenna columns (any component) from the grid's mask
    const size_t ncol = size_t(d.nx) * d.ny;
    std::vector<uint8_t> mask(ncol);
    std::vector<int> acols;
    fdtd_status st = cuda_check(cudaMemcpyAsync(mask.data(), static_cast<char*>(g->arena) + g->L.smask, ncol,
                                                cudaMemcpyDeviceToHost, g->stream), "read antenna mask");
    if (st == FDTD_OK) st = cuda_check(cudaStreamSynchronize(g->stream), "read antenna mask");
    if (st != FDTD_OK) { delete a; return st; }
    for (size_t c = 0; c < ncol; ++c)
        if (mask[c] & 0x3f) acols.push_back(int(c));
    a->nacols = int(acols.size());
    st = cuda_check(cudaMemsetAsync(arena, 0, a->dyn_bytes, g->stream), "zero adjoint");
    if (st == FDTD_OK && !acols.empty())
        st = cuda_check(cudaMemcpyAsync(static_cast<char*>(arena) + a->acols, acols.data(), acols.size() * 4,
                                        cudaMemcpyHostToDevice, g->stream), "upload antenna columns");
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
    const fdtd_status dev_st = check_device(a->g, "fdtd_adjoint_reset");
    if (dev_st != FDTD_OK) return dev_st;
    a->n = n_end;
    a->cur = 0;
    return cuda_check(cudaMemsetAsync(a->arena, 0, a->dyn_bytes, a->g->stream), "reset adjoint");
}

fdtd_status fdtd_probe_record(fdtd_adjoint* a, int nsteps, void* dev_rows, int64_t ld)
{
    if (!a || nsteps < 0 || (nsteps > 0 && !dev_rows) || ld < a->nprobes)
        return fail(FDTD_EINVAL, "fdtd_probe_record: invalid argument");
    fdtd_grid* g = a->g;
    const fdtd_status dev_st = check_device(g, "fdtd_probe_record");
    if (dev_st != FDTD_OK) return dev_st;
    if (g->batch_refs > 0) return fail(FDTD_ESTATE, "fdtd_probe_record: the grid belongs to a batch");
    const TileConfig one = single_step_tile(g->tile);
    const size_t elem = g->L.elem;
    for (int s = 0; s < nsteps; ++s) {
        cudaError_t e = launch_step(g, g->cur, g->step, one, g->stream);
        g->fault = 0;
        if (e != cudaSuccess) return cuda_check(e, "step launch");
        g->cur ^= 1;
        g->step += 1;
        if (a->nprobes > 0) {
            void* row = static_cast<char*>(dev_rows) + size_t(s) * size_t(ld) * elem;
            e = g->desc.precision == FDTD_F64 ? launch_gather<double>(a, row) : launch_gather<float>(a, row);
            if (e != cudaSuccess) return cuda_check(e, "probe gather");
        }
    }
    return FDTD_OK;
}

fdtd_status fdtd_probe_read(fdtd_adjoint* a, void* dev_out)
{
    if (!a || !dev_out) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(a->g, "fdtd_probe_read");
    if (dev_st != FDTD_OK) return dev_st;
    if (a->nprobes == 0) return FDTD_OK;
    cudaError_t e = a->g->desc.precision == FDTD_F64 ? launch_gather<double>(a, dev_out) : launch_gather<float>(a, dev_out);
    return cuda_check(e, "probe gather");
}

static fdtd_status adjoint_steps(fdtd_adjoint* a, int nsteps, const void* dLdE, int64_t ld);

fdtd_status fdtd_adjoint_step(fdtd_adjoint* a, int nsteps, const void* dLdE, int64_t ld)
{
    nvtxRangePushA("fdtd_adjoint_step");
    fdtd_status st = adjoint_steps(a, nsteps, dLdE, ld);
    nvtxRangePop();
    return st;
}

static fdtd_status adjoint_steps(fdtd_adjoint* a, int nsteps, const void* dLdE, int64_t ld)
{
    if (!a || nsteps < 0) return fail(FDTD_EINVAL, "invalid argument");
    const fdtd_status dev_st = check_device(a->g, "fdtd_adjoint_step");
    if (dev_st != FDTD_OK) return dev_st;
    if (nsteps > a->n) return fail(FDTD_EINVAL, "cannot step the adjoint before forward step 0");
    const size_t eb = a->g->L.elem;
    for (int s = 0; s < nsteps; ++s) {
        if (dLdE && a->nprobes > 0) {
            const void* row = static_cast<const char*>(dLdE) + size_t(s) * size_t(ld) * eb;
            cudaError_t e = eb == 8 ? launch_inject<double>(a, row) : launch_inject<float>(a, row);
            if (e != cudaSuccess) return cuda_check(e, "adjoint inject");
        }
        const long long n = a->n - 1;   // reverse forward step n
        cudaError_t e = eb == 8 ? adj_cell_launch<double, 4>(a, n) : adj_cell_launch<float, 4>(a, n);
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
    const fdtd_status dev_st = check_device(a->g, "fdtd_adjoint_get");
    if (dev_st != FDTD_OK) return dev_st;
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
    const fdtd_status dev_st = check_device(a->g, "fdtd_adjoint_gradient");
    if (dev_st != FDTD_OK) return dev_st;
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
