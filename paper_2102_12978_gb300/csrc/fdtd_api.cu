// fdtd_api.cu -- host side of the C ABI declared in include/fdtd.h: grid
// descriptors, arena layout, FP64 precompute of the CPML profiles (Section 4,
// Roden-Gedney CPML) and of the antenna tables (Eq. 6-9, 12, 13), kernel
// dispatch, state save/load and error reporting.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "engine.h"
#include "grid_impl.h"
#include "yee_tb2.cuh"
#include "tma_host.h"
#include "yee_fused.cuh"
#include "fluence.cuh"

namespace fdtd {

thread_local char g_last_error[512] = "";

fdtd_status fail(fdtd_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

fdtd_status cuda_check(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return FDTD_OK;
    return fail(FDTD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

fdtd_status check_device(const fdtd_grid* g, const char* what)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, what);
    if (dev != g->device)
        return fail(FDTD_EINVAL, "%s: the grid lives on device %d but device %d is current", what, g->device, dev);
    return FDTD_OK;
}

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Arena layout: the dynamic state (fields, CPML psi, fluence) first, then the
// static tables.  Every block starts on a 256-byte boundary.
bool compute_layout(const fdtd_grid_desc& d, Layout& L)
{
    const size_t b = d.precision == FDTD_F64 ? 8 : 4;
    L.elem = b;
    L.pitch = static_cast<int>(align_up(static_cast<size_t>(d.nx), 32));
    const size_t nz = d.nz, ny = d.ny, nx = d.nx, p = L.pitch, w2 = 2 * size_t(d.npml);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    L.field_elems = nz * ny * p;
    for (int buf = 0; buf < 2; ++buf)
        for (int c = 0; c < 6; ++c) L.field[buf][c] = take(L.field_elems * b);
    L.psx_elems = nz * ny * w2;
    L.psy_elems = nz * w2 * p;
    for (int buf = 0; buf < 2; ++buf)
        for (int c = 0; c < 2; ++c) {
            L.phx[buf][c] = take(L.psx_elems * b);
            L.phy[buf][c] = take(L.psy_elems * b);
        }
    for (int buf = 0; buf < 2; ++buf)
        for (int c = 0; c < 2; ++c) {
            L.pex[buf][c] = take(L.psx_elems * b);
            L.pey[buf][c] = take(L.psy_elems * b);
        }
    const size_t w2z = d.z_boundary == FDTD_Z_WALLS ? 2 * size_t(d.npml_z) : 0;
    L.psz_elems = w2z * ny * p;
    for (int buf = 0; buf < 2; ++buf)
        for (int c = 0; c < 2; ++c) L.phz[buf][c] = take(L.psz_elems * b);
    for (int c = 0; c < 2; ++c) L.pez[c] = take(L.psz_elems * b);
    L.fluence = d.fluence ? take(nz * ny * p * 8) : 0;
    L.dynamic_bytes = off;
    L.chx = take(nx * b); L.cex = take(nx * b);
    L.chy = take(ny * b); L.cey = take(ny * b);
    L.chz = take(nz * b); L.cez = take(nz * b);
    for (int q = 0; q < 8; ++q) L.prof[q] = take((w2 ? w2 : 1) * b);
    for (int q = 8; q < 12; ++q) L.prof[q] = take((w2z ? w2z : 1) * b);
    L.wcoef = take(nx * ny * 16);
    L.wcoef32 = take(nx * ny * 8);
    L.smask = take(nx * ny);
    L.scoef = take(6 * nx * ny * 16);
    L.scoef32 = take(6 * nx * ny * 8);
    L.scoef_unw = take(6 * nx * ny * 16);
    L.wamp = take(nx * ny * 8);
    L.wphase = take(nx * ny * 8);
    L.zph = take(nz * 16);
    L.zph32 = take(nz * 8);
    L.flu_out = d.fluence ? take(nz * ny * nx * 8) : 0;
    L.alist = take(2 * nx * ny * 4);
    L.tb2prof = take(size_t(kTb2MaxCtas) * 8);   // per-CTA cycles of variant 7's measuring launches
    L.err = take(256);
    L.total = off;
    return true;
}

fdtd_status validate(const fdtd_grid_desc* d)
{
    if (!d) return fail(FDTD_EINVAL, "null grid descriptor");
    if (d->nx < 2 || d->ny < 2 || d->nz < 1)
        return fail(FDTD_EINVAL, "grid %dx%dx%d too small", d->nx, d->ny, d->nz);
    if (d->npml < 0 || (d->npml > 0 && (4 * d->npml > d->nx || 4 * d->npml > d->ny)))
        return fail(FDTD_EINVAL, "npml=%d must be >= 0 and at most a quarter of nx, ny", d->npml);
    if (!(d->dx > 0) || !(d->dy > 0) || !(d->dz > 0))
        return fail(FDTD_EINVAL, "cell sizes must be positive");
    if (d->precision != FDTD_F32 && d->precision != FDTD_F64)
        return fail(FDTD_EINVAL, "unknown precision %d", d->precision);
    if (double(d->nz) * d->ny * (d->nx + 31) >= 2147483647.0)
        return fail(FDTD_EINVAL, "grid of %d x %d x %d cells exceeds the 2^31-element limit of one array",
                    d->nx, d->ny, d->nz);
    double lim = 1.0 / std::sqrt(1.0 / (d->dx * d->dx) + 1.0 / (d->dy * d->dy) + 1.0 / (d->dz * d->dz));
    if (d->dt == 0.0) {
        if (!(d->courant > 0.0) || d->courant > 1.0)
            return fail(FDTD_EINVAL, "courant=%g must be in (0, 1]", d->courant);
    } else if (!(d->dt > 0.0) || d->dt > lim) {
        return fail(FDTD_EINVAL, "dt=%g outside (0, %g] (Yee stability limit)", d->dt, lim);
    }
    if (d->z_boundary != FDTD_Z_PERIODIC && d->z_boundary != FDTD_Z_WALLS)
        return fail(FDTD_EINVAL, "z_boundary=%d is neither FDTD_Z_PERIODIC nor FDTD_Z_WALLS", d->z_boundary);
    if (d->z_boundary == FDTD_Z_PERIODIC && d->npml_z != 0)
        return fail(FDTD_EINVAL, "npml_z=%d on a z-periodic grid", d->npml_z);
    if (d->z_boundary == FDTD_Z_WALLS) {
        if (d->npml_z < 0 || 2 * d->npml_z + 2 > d->nz)
            return fail(FDTD_EINVAL, "npml_z=%d must be >= 0 with 2*npml_z + 2 <= nz=%d", d->npml_z, d->nz);
    }
    if ((d->npml > 0 || d->npml_z > 0) &&
        !(d->pml_order >= 0.0 && d->pml_sigma_scale >= 0.0 && d->pml_kappa_max >= 1.0 && d->pml_alpha_max >= 0.0))
        return fail(FDTD_EINVAL, "invalid CPML constants");
    return FDTD_OK;
}

double grid_dt(const fdtd_grid_desc& d)
{
    if (d.dt != 0.0) return d.dt;
    return d.courant / std::sqrt(1.0 / (d.dx * d.dx) + 1.0 / (d.dy * d.dy) + 1.0 / (d.dz * d.dz));
}

// CPML grading along one axis (Roden-Gedney CFS-PML; constants documented in
// fdtd_grid_desc).  For a position `pos` (cells from the low face) returns
// b, a and kappa of the auxiliary recursion psi <- b psi + a d(field)/d(axis).
static void cpml_at(const fdtd_grid_desc& d, int n, int npml, double cell, double dt, double pos_cells,
                    double& b, double& a, double& kappa)
{
    b = 1.0; a = 0.0; kappa = 1.0;
    if (npml <= 0) return;
    double depth_cells = 0.0;
    if (pos_cells < npml) depth_cells = npml - pos_cells;
    else if (pos_cells > n - npml) depth_cells = pos_cells - (n - npml);
    if (depth_cells <= 0.0) return;
    double u = depth_cells / npml;
    double grade = std::pow(u, d.pml_order);
    double sigma = d.pml_sigma_scale * (d.pml_order + 1.0) / cell * grade;
    kappa = 1.0 + (d.pml_kappa_max - 1.0) * grade;
    double alpha = d.pml_alpha_max * (1.0 - u);
    b = std::exp(-(sigma / kappa + alpha) * dt);
    if (sigma > 0.0) a = sigma * (b - 1.0) / (kappa * (sigma + kappa * alpha));
}

// Per-position coefficients dt / (kappa d) of one axis (H at i+1/2, E at i)
// and the CPML b, a' = dt a / d on its 2 npml shell positions.
template <typename real>
static void build_axis_tables(const fdtd_grid_desc& d, int n, int npml, double cell, double dt,
                              std::vector<real>& ch, std::vector<real>& ce,
                              std::vector<real>& bh, std::vector<real>& ah,
                              std::vector<real>& be, std::vector<real>& ae)
{
    const int w2 = 2 * npml;
    ch.assign(n, real(0)); ce.assign(n, real(0));
    bh.assign(w2 ? w2 : 1, real(1)); ah.assign(w2 ? w2 : 1, real(0));
    be.assign(w2 ? w2 : 1, real(1)); ae.assign(w2 ? w2 : 1, real(0));
    for (int i = 0; i < n; ++i) {
        double b, a, kap;
        cpml_at(d, n, npml, cell, dt, i + 0.5, b, a, kap);      // H sits half a cell in
        ch[i] = real(dt / (kap * cell));
        int sh = (i < npml) ? i : (i >= n - npml ? i - n + w2 : -1);
        if (sh >= 0) { bh[sh] = real(b); ah[sh] = real(dt * a / cell); }
        cpml_at(d, n, npml, cell, dt, double(i), b, a, kap);    // E on the integer position
        ce[i] = real(dt / (kap * cell));
        if (sh >= 0) { be[sh] = real(b); ae[sh] = real(dt * a / cell); }
    }
}

template <typename real>
static fdtd_status upload_tables(fdtd_grid* g)
{
    std::vector<real> chx, cex, bhx, ahx, bex, aex, chy, cey, bhy, ahy, bey, aey, chz, cez, bhz, ahz, bez, aez;
    const fdtd_grid_desc& d = g->desc;
    build_axis_tables<real>(d, d.nx, d.npml, d.dx, g->dt, chx, cex, bhx, ahx, bex, aex);
    build_axis_tables<real>(d, d.ny, d.npml, d.dy, g->dt, chy, cey, bhy, ahy, bey, aey);
    const int npz = d.z_boundary == FDTD_Z_WALLS ? d.npml_z : 0;
    build_axis_tables<real>(d, d.nz, npz, d.dz, g->dt, chz, cez, bhz, ahz, bez, aez);
    char* A = static_cast<char*>(g->arena);
    cudaStream_t s = g->stream;
    const Layout& L = g->L;
    struct { size_t off; const std::vector<real>* v; } items[] = {
        {L.chx, &chx}, {L.cex, &cex}, {L.chy, &chy}, {L.cey, &cey},
        {L.prof[0], &bhx}, {L.prof[1], &ahx}, {L.prof[2], &bex}, {L.prof[3], &aex},
        {L.prof[4], &bhy}, {L.prof[5], &ahy}, {L.prof[6], &bey}, {L.prof[7], &aey},
        {L.chz, &chz}, {L.cez, &cez},
        {L.prof[8], &bhz}, {L.prof[9], &ahz}, {L.prof[10], &bez}, {L.prof[11], &aez},
    };
    for (auto& it : items) {
        fdtd_status st = cuda_check(cudaMemcpyAsync(A + it.off, it.v->data(), it.v->size() * sizeof(real),
                                                    cudaMemcpyHostToDevice, s), "upload CPML tables");
        if (st != FDTD_OK) return st;
    }
    return cuda_check(cudaStreamSynchronize(s), "upload CPML tables");
}

template <typename real>
StepArgs<real> make_args(const fdtd_grid* g, int cur)
{
    StepArgs<real> a;
    const Layout& L = g->L;
    char* A = static_cast<char*>(g->arena);
    const int nxt = cur ^ 1;
    a.nx = g->desc.nx; a.ny = g->desc.ny; a.nz = g->desc.nz; a.npml = g->desc.npml; a.pitch = L.pitch;
    for (int c = 0; c < 3; ++c) {
        a.ein[c] = reinterpret_cast<const real*>(A + L.field[cur][c]);
        a.eout[c] = reinterpret_cast<real*>(A + L.field[nxt][c]);
        a.hin[c] = reinterpret_cast<const real*>(A + L.field[cur][3 + c]);
        a.hout[c] = reinterpret_cast<real*>(A + L.field[nxt][3 + c]);
    }
    for (int c = 0; c < 2; ++c) {
        a.phx_in[c] = reinterpret_cast<const real*>(A + L.phx[cur][c]);
        a.phx_out[c] = reinterpret_cast<real*>(A + L.phx[nxt][c]);
        a.phy_in[c] = reinterpret_cast<const real*>(A + L.phy[cur][c]);
        a.phy_out[c] = reinterpret_cast<real*>(A + L.phy[nxt][c]);
        a.pex[c] = reinterpret_cast<real*>(A + L.pex[g->pe][c]);
        a.pey[c] = reinterpret_cast<real*>(A + L.pey[g->pe][c]);
        a.pex_out[c] = reinterpret_cast<real*>(A + L.pex[g->pe ^ 1][c]);
        a.pey_out[c] = reinterpret_cast<real*>(A + L.pey[g->pe ^ 1][c]);
    }
    a.chx = reinterpret_cast<const real*>(A + L.chx);
    a.cex = reinterpret_cast<const real*>(A + L.cex);
    a.chy = reinterpret_cast<const real*>(A + L.chy);
    a.cey = reinterpret_cast<const real*>(A + L.cey);
    a.bhx = reinterpret_cast<const real*>(A + L.prof[0]);
    a.ahx = reinterpret_cast<const real*>(A + L.prof[1]);
    a.bex = reinterpret_cast<const real*>(A + L.prof[2]);
    a.aex = reinterpret_cast<const real*>(A + L.prof[3]);
    a.bhy = reinterpret_cast<const real*>(A + L.prof[4]);
    a.ahy = reinterpret_cast<const real*>(A + L.prof[5]);
    a.bey = reinterpret_cast<const real*>(A + L.prof[6]);
    a.aey = reinterpret_cast<const real*>(A + L.prof[7]);
    a.cz = real(g->dt / g->desc.dz);
    a.dt = g->dt;
    a.dt16 = g->dt * 0.0625;
    a.fluence = g->desc.fluence ? static_cast<void*>(A + L.fluence) : nullptr;
    a.smask = g->has_source ? reinterpret_cast<const uint8_t*>(A + L.smask) : nullptr;
    a.scoef = reinterpret_cast<const double2*>(A + L.scoef);
    a.scoefr = sizeof(real) == 8 ? static_cast<const void*>(A + L.scoef) : static_cast<const void*>(A + L.scoef32);
    a.zph = reinterpret_cast<const double2*>(A + L.zph);
    a.zphr = sizeof(real) == 8 ? static_cast<const void*>(A + L.zph) : static_cast<const void*>(A + L.zph32);
    a.st = g->srct;
    a.fault = g->fault;
    a.zw = g->desc.z_boundary == FDTD_Z_WALLS;
    a.npz = a.zw ? g->desc.npml_z : 0;
    for (int c = 0; c < 2; ++c) {
        a.phz_in[c] = reinterpret_cast<const real*>(A + L.phz[cur][c]);
        a.phz_out[c] = reinterpret_cast<real*>(A + L.phz[nxt][c]);
        a.pez[c] = reinterpret_cast<real*>(A + L.pez[c]);
    }
    a.chz = reinterpret_cast<const real*>(A + L.chz);
    a.cez = reinterpret_cast<const real*>(A + L.cez);
    a.bhz = reinterpret_cast<const real*>(A + L.prof[8]);
    a.ahz = reinterpret_cast<const real*>(A + L.prof[9]);
    a.bez = reinterpret_cast<const real*>(A + L.prof[10]);
    a.aez = reinterpret_cast<const real*>(A + L.prof[11]);
    a.wcoefr = !g->has_wall ? nullptr
               : sizeof(real) == 8 ? static_cast<const void*>(A + L.wcoef) : static_cast<const void*>(A + L.wcoef32);
    a.wplane = g->has_wall ? g->wall.plane : -1;
    a.kbase = 0;
    return a;
}

template StepArgs<float> make_args<float>(const fdtd_grid*, int);
template StepArgs<double> make_args<double>(const fdtd_grid*, int);

// ---- kernel dispatch over (variant, precision, tile)
template <typename real, int TX, int TY>
static cudaError_t launch_fused(const fdtd_grid* g, int cur, long long n, int lz, cudaStream_t s)
{
    using T = FusedTile<real, TX, TY>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(yee_step_fused<real, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(T::smem_bytes()));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 block(TX, TY);
    dim3 grid((g->desc.nx + TX - 1) / TX, (g->desc.ny + TY - 1) / TY, (g->desc.nz + lz - 1) / lz);
    yee_step_fused<real, TX, TY><<<grid, block, T::smem_bytes(), s>>>(make_args<real>(g, cur), n, lz);
    return cudaGetLastError();
}

// 32 x TR tiles, R rows per thread (32 x TR/R threads), S stages.
template <typename real, int TR, int R, int S>
static cudaError_t launch_tma(const fdtd_grid* cg, int cur, long long n, int lz, cudaStream_t s)
{
    fdtd_grid* g = const_cast<fdtd_grid*>(cg);
    using T = TmaTile<real, TR>;
    const size_t smem = T::smem_bytes(S, lz);
    static size_t attr_set = 0;
    if (smem > attr_set) {
        cudaError_t e = cudaFuncSetAttribute(yee_step_tma<real, TR, R, S>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        attr_set = smem;
    }
    TmaMaps* m = nullptr;
    if (!tma_maps<real, TR>(g, cur, &m)) return cudaErrorInvalidValue;
    dim3 block(32, TR / R);
    dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TR - 1) / TR, (g->desc.nz + lz - 1) / lz);
    int* err = reinterpret_cast<int*>(static_cast<char*>(g->arena) + g->L.err);
    yee_step_tma<real, TR, R, S><<<grid, block, smem, s>>>(make_args<real>(g, cur), *m, n, lz, err);
    return cudaGetLastError();
}

cudaError_t launch_step(const fdtd_grid* g, int cur, long long n, const TileConfig& tc, cudaStream_t s,
                        cudaEvent_t mid)
{
    if (tc.variant != 5 && needs_cell_passes(g)) return cudaErrorInvalidValue;   // z walls / wall source
    if (tc.variant == 7) return cudaErrorInvalidValue;   // two steps per launch: launch_tb2
    if (tc.variant >= 3) return launch_split(g, cur, n, tc, s, mid);   // variants 3-6
    if (tc.variant == 1) {
        if (g->desc.precision == FDTD_F32) {
            switch (tc.ty) {
                case 4: return launch_tma<float, 4, 1, 6>(g, cur, n, tc.lz, s);
                case 16: return launch_tma<float, 16, 1, 5>(g, cur, n, tc.lz, s);
                default: return launch_tma<float, 8, 1, 5>(g, cur, n, tc.lz, s);
            }
        } else {
            switch (tc.ty) {
                case 4: return launch_tma<double, 4, 1, 5>(g, cur, n, tc.lz, s);
                default: return launch_tma<double, 8, 1, 5>(g, cur, n, tc.lz, s);
            }
        }
    }
    if (tc.variant == 2) {
        if (g->desc.precision == FDTD_F32) {
            switch (tc.ty) {
                case 4: return launch_tma<float, 4, 2, 6>(g, cur, n, tc.lz, s);
                case 16: return launch_tma<float, 16, 2, 5>(g, cur, n, tc.lz, s);
                default: return launch_tma<float, 8, 2, 5>(g, cur, n, tc.lz, s);
            }
        } else {
            switch (tc.ty) {
                case 4: return launch_tma<double, 4, 2, 5>(g, cur, n, tc.lz, s);
                default: return launch_tma<double, 8, 2, 5>(g, cur, n, tc.lz, s);
            }
        }
    }
    if (g->desc.precision == FDTD_F32) {
        switch (tc.ty) {
            case 4: return launch_fused<float, 32, 4>(g, cur, n, tc.lz, s);
            case 16: return launch_fused<float, 32, 16>(g, cur, n, tc.lz, s);
            default: return launch_fused<float, 32, 8>(g, cur, n, tc.lz, s);
        }
    } else {
        switch (tc.ty) {
            case 4: return launch_fused<double, 32, 4>(g, cur, n, tc.lz, s);
            case 16: return launch_fused<double, 32, 16>(g, cur, n, tc.lz, s);
            default: return launch_fused<double, 32, 8>(g, cur, n, tc.lz, s);
        }
    }
}

// Default tile: the cell-parallel two-pass step on 32 x 4 blocks (the
// fastest on GB300 for every grid measured; grids of more than 65535 planes
// are launched in chunks of planes).
TileConfig default_tile(const fdtd_grid_desc& d, int sm_count)
{
    (void)sm_count;
    TileConfig tc;
    tc.variant = 5; tc.tx = 32; tc.ty = 4; tc.lz = d.nz;
    return tc;
}

}  // namespace fdtd

using namespace fdtd;

extern "C" {

void fdtd_grid_desc_default(fdtd_grid_desc* d)
{
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->courant = 0.95;
    d->pml_order = 3.0;
    d->pml_sigma_scale = 0.8;
    d->pml_kappa_max = 1.0;
    d->pml_alpha_max = 0.05 * 2.0 * M_PI;
    d->precision = FDTD_F32;
    d->fluence = 1;
}

size_t fdtd_required_bytes(const fdtd_grid_desc* d)
{
    if (validate(d) != FDTD_OK) return 0;
    Layout L;
    compute_layout(*d, L);
    return L.total;
}

fdtd_status fdtd_create_grid(const fdtd_grid_desc* d, void* arena, size_t arena_bytes, void* stream,
                             fdtd_grid** out)
{
    if (!out) return fail(FDTD_EINVAL, "null output pointer");
    *out = nullptr;
    fdtd_status st = validate(d);
    if (st != FDTD_OK) return st;
    if (!arena) return fail(FDTD_EINVAL, "null arena");
    if (reinterpret_cast<uintptr_t>(arena) % 256 != 0) return fail(FDTD_EINVAL, "arena not 256-byte aligned");
    Layout L;
    compute_layout(*d, L);
    if (arena_bytes < L.total)
        return fail(FDTD_ENOMEM, "arena of %zu bytes, %zu needed", arena_bytes, L.total);
    fdtd_grid* g = new (std::nothrow) fdtd_grid();
    if (!g) return fail(FDTD_ENOMEM, "host allocation failed");
    g->desc = *d;
    g->L = L;
    g->arena = arena;
    g->arena_bytes = arena_bytes;
    g->stream = static_cast<cudaStream_t>(stream);
    g->dt = grid_dt(*d);
    g->step = 0;
    g->cur = 0;
    g->pe = 0;
    g->has_source = false;
    g->src_gen = 0;
    g->tb2_key.ry = 0;
    g->tb2_ref_ry = 0;
    g->tb2_ref_slots = 0;
    g->tb2_ref_src = -1;
    g->tb2_ref_order = 0;
    g->tb2_ref_gen = 0;
    g->tb2_profile = false;
    g->ant_cols[0] = g->ant_cols[1] = 0;
    g->ant_apart = false;
    std::memset(&g->srct, 0, sizeof(g->srct));
    g->srct.dt = g->dt;
    g->batch_refs = 0;
    g->has_wall = false;
    std::memset(&g->wall, 0, sizeof(g->wall));
    std::memset(&g->wallt, 0, sizeof(g->wallt));
    g->fault = 0;
    for (int c = 0; c < 6; ++c) g->counts[c] = 0;
    int dev = 0, sms = 152;
    st = cuda_check(cudaGetDevice(&dev), "current device");
    if (st != FDTD_OK) { delete g; return st; }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g->sm_count = sms;
    g->device = dev;
    st = noalloc_prepare(dev);
    if (st != FDTD_OK) { delete g; return st; }
    g->tile = default_tile(*d, sms);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) g->maps_ok[a][b] = g->hmaps_ok[a][b] = false;
    st = cuda_check(cudaMemsetAsync(arena, 0, L.total, g->stream), "zero arena");
    if (st == FDTD_OK)
        st = (d->precision == FDTD_F64) ? upload_tables<double>(g) : upload_tables<float>(g);
    if (st != FDTD_OK) { delete g; return st; }
    *out = g;
    return FDTD_OK;
}

// Checks of an annulus descriptor against its grid (EINVAL with a message).
static fdtd_status validate_source(const fdtd_grid_desc& d, const fdtd_annulus_desc* s)
{
    if (d.z_boundary != FDTD_Z_PERIODIC)
        return fail(FDTD_EINVAL, "the antenna takes z-periodic grids (Section 4); this grid has z walls");
    if (s->pol < FDTD_POL_Y || s->pol > FDTD_POL_Z || (s->mode != FDTD_TE && s->mode != FDTD_TM) ||
        (s->envelope != FDTD_ENV_CW_SIN2 && s->envelope != FDTD_ENV_GAUSS) ||
        (s->inject != FDTD_INJECT_ALL && s->inject != FDTD_INJECT_TANGENTIAL))
        return fail(FDTD_EINVAL, "invalid enum in annulus descriptor");
    if (!(s->thickness > 0.0) || !(s->r_center > 0.5 * s->thickness))
        return fail(FDTD_EINVAL, "ring thickness %g / radius %g invalid", s->thickness, s->r_center);
    double rout = s->r_center + 0.5 * s->thickness;
    double room = std::min(0.5 * d.nx, 0.5 * d.ny) - d.npml - 1.0;
    if (rout > room)
        return fail(FDTD_EINVAL, "ring outer radius %g cells reaches the CPML (limit %g)", rout, room);
    if (s->envelope == FDTD_ENV_GAUSS && !(s->T > 0.0)) return fail(FDTD_EINVAL, "Gaussian T must be > 0");
    if (s->envelope == FDTD_ENV_CW_SIN2 && s->ramp < 0.0) return fail(FDTD_EINVAL, "ramp must be >= 0");
    return FDTD_OK;
}

// Calls that change what a batch captured, or step the grid by itself, are
// refused while the grid belongs to a batch.
static fdtd_status not_batched(const fdtd_grid* g, const char* what)
{
    if (g->batch_refs > 0) return fail(FDTD_ESTATE, "%s: the grid belongs to a batch", what);
    return FDTD_OK;
}

fdtd_status fdtd_set_annulus_source(fdtd_grid* g, const fdtd_annulus_desc* s)
{
    if (!g || !s) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(g, "fdtd_set_annulus_source");
    if (dev_st != FDTD_OK) return dev_st;
    if (g->batch_refs > 0) return not_batched(g, "fdtd_set_annulus_source");
    const fdtd_grid_desc& d = g->desc;
    fdtd_status vst = validate_source(d, s);
    if (vst != FDTD_OK) return vst;
    GridSpec gs{d.nx, d.ny, d.nz, d.npml, d.dx, d.dy, d.dz, g->dt};
    SourceSpec ss{s->m, s->theta, s->pol, s->mode, s->E0, s->r_center, s->thickness, s->inject};
    std::vector<std::complex<double>> coef, coef_unw;
    std::vector<uint8_t> mask;
    int64_t counts[6];
    source_tables(gs, ss, nullptr, nullptr, coef_unw, mask, counts);
    const size_t ncol = size_t(d.nx) * d.ny;
    std::vector<double> wamp(ncol, 1.0), wph(ncol, 0.0);
    if (s->w_amp) std::memcpy(wamp.data(), s->w_amp, ncol * 8);
    if (s->w_phase) std::memcpy(wph.data(), s->w_phase, ncol * 8);
    coef.resize(coef_unw.size());
    for (size_t q = 0; q < coef_unw.size(); ++q) coef[q] = std::polar(wamp[q % ncol], wph[q % ncol]) * coef_unw[q];
    // e^{i beta k dz}: the coefficients already carry each component's own
    // half-cell z offset, so one table serves every component
    const double beta = 2.0 * M_PI * std::cos(s->theta);
    std::vector<std::complex<double>> zph(size_t(d.nz));
    for (int k = 0; k < d.nz; ++k) zph[k] = std::polar(1.0, beta * (k * d.dz));
    char* A = static_cast<char*>(g->arena);
    fdtd_status st = cuda_check(cudaMemcpyAsync(A + g->L.scoef, coef.data(), coef.size() * 16,
                                                cudaMemcpyHostToDevice, g->stream), "upload source");
    std::vector<float> coef32(2 * coef.size());
    for (size_t q = 0; q < coef.size(); ++q) {
        coef32[2 * q] = float(coef[q].real());
        coef32[2 * q + 1] = float(coef[q].imag());
    }
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.scoef32, coef32.data(), coef32.size() * 4, cudaMemcpyHostToDevice,
                                        g->stream), "upload source");
    // device copy of the mask: bit 6 marks the columns whose own or +-x / +-y
    // neighbour column carries an H antenna point (the one-pass cell kernel
    // evaluates H source terms of recomputed neighbours only there)
    std::vector<uint8_t> dmask(mask);
    for (int j = 0; j < d.ny; ++j)
        for (int i = 0; i < d.nx; ++i) {
            auto hbits = [&](int ii, int jj) {
                return ii >= 0 && ii < d.nx && jj >= 0 && jj < d.ny && (mask[size_t(jj) * d.nx + ii] & 0x38);
            };
            if (hbits(i, j) || hbits(i - 1, j) || hbits(i + 1, j) || hbits(i, j - 1) || hbits(i, j + 1))
                dmask[size_t(j) * d.nx + i] |= 0x40;
        }
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.smask, dmask.data(), dmask.size(), cudaMemcpyHostToDevice,
                                        g->stream), "upload source");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.scoef_unw, coef_unw.data(), coef_unw.size() * 16,
                                        cudaMemcpyHostToDevice, g->stream), "upload source");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.wamp, wamp.data(), ncol * 8, cudaMemcpyHostToDevice, g->stream),
                        "upload source");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.wphase, wph.data(), ncol * 8, cudaMemcpyHostToDevice, g->stream),
                        "upload source");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.zph, zph.data(), zph.size() * 16, cudaMemcpyHostToDevice,
                                        g->stream), "upload source");
    std::vector<float> zph32(2 * zph.size());
    for (size_t q = 0; q < zph.size(); ++q) {
        zph32[2 * q] = float(zph[q].real());
        zph32[2 * q + 1] = float(zph[q].imag());
    }
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.zph32, zph32.data(), zph32.size() * 4, cudaMemcpyHostToDevice,
                                        g->stream), "upload source");
    // the antenna's columns as two lists (H points, E points) for antenna_add
    std::vector<int> alist;
    int ncol_h = 0;
    bool on_wall = false;
    for (int side = 0; side < 2; ++side)
        for (int j = 0; j < d.ny; ++j)
            for (int i = 0; i < d.nx; ++i) {
                const uint8_t m = mask[size_t(j) * d.nx + i] & (side == 0 ? 0x38 : 0x07);
                if (!m) continue;
                alist.push_back(j * d.nx + i);
                on_wall = on_wall || i == 0 || j == 0;
                if (side == 0) ++ncol_h;
            }
    if (st == FDTD_OK && !alist.empty())
        st = cuda_check(cudaMemcpyAsync(A + g->L.alist, alist.data(), alist.size() * 4, cudaMemcpyHostToDevice,
                                        g->stream), "upload source");
    if (st == FDTD_OK) st = cuda_check(cudaStreamSynchronize(g->stream), "upload source");
    if (st != FDTD_OK) return st;
    g->ant_cols[0] = ncol_h;
    g->ant_cols[1] = int(alist.size()) - ncol_h;
    g->ant_apart = !on_wall;
    g->has_source = true;
    if (mask != g->hmask) g->src_gen += 1;   // the antenna's columns changed
    g->hmask = mask;
    g->src = *s;
    g->src.w_amp = nullptr;
    g->src.w_phase = nullptr;
    g->srct.gauss = s->envelope == FDTD_ENV_GAUSS;
    g->srct.ramp = s->ramp;
    g->srct.T = s->T;
    g->srct.T0 = s->T0;
    g->srct.dt = g->dt;
    for (int c = 0; c < 6; ++c) g->counts[c] = counts[c];
    return FDTD_OK;
}

// Checks of a wall-source descriptor against its grid (EINVAL with a message).
static fdtd_status validate_wall(const fdtd_grid_desc& d, const fdtd_wall_desc* w)
{
    if (w->envelope != FDTD_ENV_CW_SIN2 && w->envelope != FDTD_ENV_GAUSS)
        return fail(FDTD_EINVAL, "invalid envelope %d in wall descriptor", w->envelope);
    if (!(w->w0 > 0.0) || !std::isfinite(w->w0)) return fail(FDTD_EINVAL, "wall waist w0=%g must be > 0", w->w0);
    if (!std::isfinite(w->theta) || !std::isfinite(w->E0)) return fail(FDTD_EINVAL, "wall theta / E0 not finite");
    if (w->plane < 0 || w->plane >= d.nz) return fail(FDTD_EINVAL, "wall plane %d outside [0, %d)", w->plane, d.nz);
    if (d.z_boundary == FDTD_Z_WALLS && w->plane == 0)
        return fail(FDTD_EINVAL, "wall plane 0 is the z = 0 PEC wall");
    if (w->envelope == FDTD_ENV_GAUSS && !(w->T > 0.0)) return fail(FDTD_EINVAL, "Gaussian T must be > 0");
    if (w->envelope == FDTD_ENV_CW_SIN2 && w->ramp < 0.0) return fail(FDTD_EINVAL, "ramp must be >= 0");
    return FDTD_OK;
}

// Column coefficients of the wall source (Section 2: Gaussian waist times the
// axicon phase -k r sin(theta), k = 2 pi) at the E_x points (i+1/2, j) of a
// plane, FP64; the row j = 0 lies on the y = 0 PEC wall and stays zero.
static void wall_tables(const fdtd_grid_desc& d, const fdtd_wall_desc* w, std::vector<std::complex<double>>& W)
{
    W.assign(size_t(d.nx) * d.ny, std::complex<double>(0.0, 0.0));
    const double kr = 2.0 * M_PI * std::sin(w->theta);
    const double xc = 0.5 * d.nx * d.dx, yc = 0.5 * d.ny * d.dy;
    for (int j = 1; j < d.ny; ++j)
        for (int i = 0; i < d.nx; ++i) {
            const double x = (i + 0.5) * d.dx - xc, y = j * d.dy - yc;
            const double r = std::sqrt(x * x + y * y);
            W[size_t(j) * d.nx + i] = std::polar(w->E0 * std::exp(-(r * r) / (w->w0 * w->w0)), -kr * r);
        }
}

fdtd_status fdtd_set_wall_source(fdtd_grid* g, const fdtd_wall_desc* w)
{
    if (!g) return fail(FDTD_EINVAL, "null grid");
    const fdtd_status dev_st = check_device(g, "fdtd_set_wall_source");
    if (dev_st != FDTD_OK) return dev_st;
    if (g->batch_refs > 0) return not_batched(g, "fdtd_set_wall_source");
    if (!w) {
        g->has_wall = false;
        return FDTD_OK;
    }
    fdtd_status st = validate_wall(g->desc, w);
    if (st != FDTD_OK) return st;
    if (g->tile.variant != 5)
        return fail(FDTD_EINVAL, "the wall source runs on tile variant 5 (this grid: %d)", g->tile.variant);
    std::vector<std::complex<double>> W;
    wall_tables(g->desc, w, W);
    std::vector<float> W32(2 * W.size());
    for (size_t q = 0; q < W.size(); ++q) {
        W32[2 * q] = float(W[q].real());
        W32[2 * q + 1] = float(W[q].imag());
    }
    char* A = static_cast<char*>(g->arena);
    st = cuda_check(cudaMemcpyAsync(A + g->L.wcoef, W.data(), W.size() * 16, cudaMemcpyHostToDevice, g->stream),
                    "upload wall source");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(A + g->L.wcoef32, W32.data(), W32.size() * 4, cudaMemcpyHostToDevice,
                                        g->stream), "upload wall source");
    if (st == FDTD_OK) st = cuda_check(cudaStreamSynchronize(g->stream), "upload wall source");
    if (st != FDTD_OK) return st;
    g->has_wall = true;
    g->wall = *w;
    g->wallt.gauss = w->envelope == FDTD_ENV_GAUSS;
    g->wallt.ramp = w->ramp;
    g->wallt.T = w->T;
    g->wallt.T0 = w->T0;
    g->wallt.dt = g->dt;
    return FDTD_OK;
}

fdtd_status fdtd_wall_coefficients(const fdtd_grid_desc* d, const fdtd_wall_desc* w, double* out)
{
    fdtd_status st = validate(d);
    if (st != FDTD_OK) return st;
    if (!w || !out) return fail(FDTD_EINVAL, "null argument");
    st = validate_wall(*d, w);
    if (st != FDTD_OK) return st;
    std::vector<std::complex<double>> W;
    wall_tables(*d, w, W);
    std::memcpy(out, W.data(), W.size() * 16);
    return FDTD_OK;
}

fdtd_status fdtd_clear_source(fdtd_grid* g)
{
    if (!g) return fail(FDTD_EINVAL, "null grid");
    if (g->batch_refs > 0) return not_batched(g, "fdtd_clear_source");
    g->has_source = false;
    g->hmask.clear();
    g->ant_cols[0] = g->ant_cols[1] = 0;
    g->src_gen += 1;
    for (int c = 0; c < 6; ++c) g->counts[c] = 0;
    return FDTD_OK;
}

// Advance the grid by nsteps with tile configuration tc on its stream: pairs
// of steps as one launch of variant 7, every other step as one launch_step.
static cudaError_t run_steps(fdtd_grid* g, int nsteps, const TileConfig& tc)
{
    int s = 0;
    if (tc.variant == 7)
        for (; s + 2 <= nsteps; s += 2) {
            cudaError_t e = launch_tb2(g, g->cur, g->step, tc, g->stream);
            if (e != cudaSuccess) return e;
            g->cur ^= 1;
            g->pe ^= 1;
            g->step += 2;
        }
    const TileConfig one = single_step_tile(tc);
    for (; s < nsteps; ++s) {
        cudaError_t e = launch_step(g, g->cur, g->step, one, g->stream);
        g->fault = 0;
        if (e != cudaSuccess) return e;
        g->cur ^= 1;
        g->step += 1;
    }
    return cudaSuccess;
}

// Variant 7 in configuration tc, measured and refined kRefineRounds times:
// kMeasureLaunches launches record every CTA's SM cycles, and tb2_refine
// moves the ranges' boundaries toward equal CTA times (all the way in the
// first round, three quarters of the way after it).  Advances the grid by
// 2 kMeasureLaunches kRefineRounds steps.
constexpr int kMeasureLaunches = 3;
constexpr int kRefineRounds = 4;
static cudaError_t tb2_measure(fdtd_grid* g, const TileConfig& tc)
{
    const int slots = tb2_slots(g, tc.ty);
    if (slots <= 0) return cudaErrorInvalidConfiguration;
    void* prof = static_cast<char*>(g->arena) + g->L.tb2prof;
    TileConfig t = tc;
    for (int round = 0; round < kRefineRounds; ++round) {
        cudaError_t err = cudaMemsetAsync(prof, 0, size_t(slots) * 8, g->stream);
        if (err != cudaSuccess) return err;
        g->tb2_profile = true;
        err = run_steps(g, 2 * kMeasureLaunches, t);
        g->tb2_profile = false;
        if (err != cudaSuccess) return err;
        std::vector<unsigned long long> cycles(static_cast<size_t>(slots));
        err = cudaMemcpyAsync(cycles.data(), prof, size_t(slots) * 8, cudaMemcpyDeviceToHost, g->stream);
        if (err == cudaSuccess) err = cudaStreamSynchronize(g->stream);
        if (err != cudaSuccess) return err;
        tb2_refine(g, t.ty, slots, cycles.data(), round == 0 ? 1.0 : 0.75);
        t.measured = true;   // the next round measures the refined ranges
    }
    return cudaSuccess;
}

fdtd_status fdtd_measure_balance(fdtd_grid* g, void* scratch_state)
{
    if (!g || !scratch_state) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(g, "fdtd_measure_balance");
    if (dev_st != FDTD_OK) return dev_st;
    if (g->batch_refs > 0) return not_batched(g, "fdtd_measure_balance");
    if (g->tile.variant != 7) return fail(FDTD_EINVAL, "fdtd_measure_balance needs tile variant 7");
    fdtd_status st = fdtd_save_state(g, scratch_state);
    if (st != FDTD_OK) return st;
    TileConfig tc = g->tile;
    const cudaError_t err = tb2_measure(g, tc);
    st = fdtd_load_state(g, scratch_state);
    if (err != cudaSuccess) return cuda_check(err, "fdtd_measure_balance");
    if (st != FDTD_OK) return st;
    g->tile.measured = true;
    return FDTD_OK;
}

fdtd_status fdtd_step(fdtd_grid* g, int nsteps)
{
    if (!g) return fail(FDTD_EINVAL, "null grid");
    if (nsteps < 0) return fail(FDTD_EINVAL, "nsteps < 0");
    const fdtd_status dev_st = check_device(g, "fdtd_step");
    if (dev_st != FDTD_OK) return dev_st;
    if (g->batch_refs > 0) return not_batched(g, "fdtd_step");
    nvtxRangePushA("fdtd_step");
    const cudaError_t e = run_steps(g, nsteps, g->tile);
    g->fault = 0;
    nvtxRangePop();
    return cuda_check(e, "step launch");
}

fdtd_status fdtd_debug_inject_fault(fdtd_grid* g, int kind)
{
    if (!g) return fail(FDTD_EINVAL, "null grid");
    if (kind != 0 && kind != 1) return fail(FDTD_EINVAL, "fault kind %d not in {0, 1}", kind);
    g->fault = kind;
    return FDTD_OK;
}

fdtd_status fdtd_debug_set_device(fdtd_grid* g, int device)
{
    if (!g || device < 0) return fail(FDTD_EINVAL, "invalid argument");
    g->device = device;
    return FDTD_OK;
}

fdtd_status fdtd_step_timed(fdtd_grid* g, int nsteps, float* pass_ms, int max_passes, int* n_passes)
{
    if (!g || !pass_ms || !n_passes || nsteps < 1) return fail(FDTD_EINVAL, "invalid argument");
    const fdtd_status dev_st = check_device(g, "fdtd_step_timed");
    if (dev_st != FDTD_OK) return dev_st;
    if (g->batch_refs > 0) return not_batched(g, "fdtd_step_timed");
    if (g->tile.variant == 7) {
        // one kernel per two steps: pass_ms[0] sums the launches
        if (nsteps % 2) return fail(FDTD_EINVAL, "variant 7 times an even number of steps (%d)", nsteps);
        const int nl = nsteps / 2;
        std::vector<cudaEvent_t> ev(size_t(nl) + 1, nullptr);
        fdtd_status st = FDTD_OK;
        for (auto& e : ev)
            if (st == FDTD_OK) st = cuda_check(cudaEventCreate(&e), "event create");
        if (st == FDTD_OK) cudaEventRecord(ev[0], g->stream);
        for (int l = 0; l < nl && st == FDTD_OK; ++l) {
            st = cuda_check(launch_tb2(g, g->cur, g->step, g->tile, g->stream), "step launch");
            cudaEventRecord(ev[size_t(l) + 1], g->stream);
            if (st == FDTD_OK) { g->cur ^= 1; g->pe ^= 1; g->step += 2; }
        }
        if (st == FDTD_OK) st = cuda_check(cudaEventSynchronize(ev.back()), "event synchronize");
        pass_ms[0] = 0.0f;
        for (int l = 0; l < nl && st == FDTD_OK; ++l) {
            float ms = 0.0f;
            st = cuda_check(cudaEventElapsedTime(&ms, ev[size_t(l)], ev[size_t(l) + 1]), "event elapsed time");
            pass_ms[0] += ms;
        }
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        *n_passes = 1;
        if (st != FDTD_OK) return st;
        return fdtd_sync(g);
    }
    const int np = passes_per_step(g->tile);
    if (max_passes < np) return fail(FDTD_EINVAL, "max_passes=%d < %d kernels per step", max_passes, np);
    std::vector<cudaEvent_t> ev(size_t(nsteps) * (np + 1), nullptr);
    fdtd_status st = FDTD_OK;
    for (auto& e : ev)
        if (st == FDTD_OK) st = cuda_check(cudaEventCreate(&e), "event create");
    for (int s = 0; s < nsteps && st == FDTD_OK; ++s) {
        cudaEvent_t* e = &ev[size_t(s) * (np + 1)];
        cudaEventRecord(e[0], g->stream);
        st = cuda_check(launch_step(g, g->cur, g->step, g->tile, g->stream, np == 2 ? e[1] : nullptr), "step launch");
        g->fault = 0;
        cudaEventRecord(e[np], g->stream);
        if (st == FDTD_OK) { g->cur ^= 1; g->step += 1; }
    }
    if (st == FDTD_OK) st = cuda_check(cudaEventSynchronize(ev.back()), "event synchronize");
    for (int p = 0; p < np; ++p) pass_ms[p] = 0.0f;
    for (int s = 0; s < nsteps && st == FDTD_OK; ++s)
        for (int p = 0; p < np; ++p) {
            float ms = 0.0f;
            st = cuda_check(cudaEventElapsedTime(&ms, ev[size_t(s) * (np + 1) + p], ev[size_t(s) * (np + 1) + p + 1]),
                            "event elapsed time");
            pass_ms[p] += ms;
        }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    *n_passes = np;
    if (st != FDTD_OK) return st;
    return fdtd_sync(g);
}

fdtd_status fdtd_sync(fdtd_grid* g)
{
    if (!g) return fail(FDTD_EINVAL, "null grid");
    const fdtd_status dev_st = check_device(g, "fdtd_sync");
    if (dev_st != FDTD_OK) return dev_st;
    fdtd_status st = cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
    if (st != FDTD_OK) return st;
    st = cuda_check(cudaGetLastError(), "pending CUDA error");
    if (st != FDTD_OK) return st;
    int err = 0;
    st = cuda_check(cudaMemcpy(&err, static_cast<char*>(g->arena) + g->L.err, sizeof(int), cudaMemcpyDeviceToHost),
                    "read error word");
    if (st != FDTD_OK) return st;
    if (err != 0) {
        cudaMemsetAsync(static_cast<char*>(g->arena) + g->L.err, 0, sizeof(int), g->stream);
        cudaStreamSynchronize(g->stream);
        return fail(FDTD_ETIMEOUT, "a bounded device-side wait expired (error word %d)", err);
    }
    return FDTD_OK;
}

fdtd_status fdtd_fluence(fdtd_grid* g, void* dst, int on_device, int reset)
{
    if (!g || !dst) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(g, "fdtd_fluence");
    if (dev_st != FDTD_OK) return dev_st;
    if (!g->desc.fluence) return fail(FDTD_ESTATE, "grid created without a fluence accumulator");
    const fdtd_grid_desc& d = g->desc;
    char* A = static_cast<char*>(g->arena);
    double* out = reinterpret_cast<double*>(A + g->L.flu_out);
    int blocks = 4 * (g->sm_count > 0 ? g->sm_count : 152);
    if (d.precision == FDTD_F64)
        fluence_export<double><<<blocks, 256, 0, g->stream>>>(reinterpret_cast<const double*>(A + g->L.fluence),
                                                              out, d.nx, d.ny, d.nz, g->L.pitch, 1.0);
    else
        fluence_export<float2><<<blocks, 256, 0, g->stream>>>(reinterpret_cast<const float2*>(A + g->L.fluence),
                                                               out, d.nx, d.ny, d.nz, g->L.pitch, 1.0);
    fdtd_status st = cuda_check(cudaGetLastError(), "fluence_export launch");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(dst, out, size_t(d.nx) * d.ny * d.nz * 8,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream),
                        "copy fluence");
    if (st == FDTD_OK && reset)
        st = cuda_check(cudaMemsetAsync(A + g->L.fluence, 0, g->L.field_elems * 8, g->stream), "reset fluence");
    if (st != FDTD_OK) return st;
    return fdtd_sync(g);
}

fdtd_status fdtd_get_field(fdtd_grid* g, int component, void* dst, int on_device)
{
    if (!g || !dst) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(g, "fdtd_get_field");
    if (dev_st != FDTD_OK) return dev_st;
    if (component < 0 || component > 5) return fail(FDTD_EINVAL, "component %d out of range", component);
    const fdtd_grid_desc& d = g->desc;
    const size_t b = g->L.elem;
    char* A = static_cast<char*>(g->arena);
    fdtd_status st = cuda_check(
        cudaMemcpy2DAsync(dst, size_t(d.nx) * b, A + g->L.field[g->cur][component], size_t(g->L.pitch) * b,
                          size_t(d.nx) * b, size_t(d.ny) * d.nz,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream),
        "copy field");
    if (st != FDTD_OK) return st;
    return fdtd_sync(g);
}

fdtd_status fdtd_set_field(fdtd_grid* g, int component, const void* src, int on_device)
{
    if (!g || !src) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(g, "fdtd_set_field");
    if (dev_st != FDTD_OK) return dev_st;
    if (component < 0 || component > 5) return fail(FDTD_EINVAL, "component %d out of range", component);
    const fdtd_grid_desc& d = g->desc;
    const size_t b = g->L.elem;
    char* A = static_cast<char*>(g->arena);
    fdtd_status st = cuda_check(
        cudaMemcpy2DAsync(A + g->L.field[g->cur][component], size_t(g->L.pitch) * b, src, size_t(d.nx) * b,
                          size_t(d.nx) * b, size_t(d.ny) * d.nz,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream),
        "set field");
    if (st != FDTD_OK) return st;
    return fdtd_sync(g);
}

size_t fdtd_state_bytes(const fdtd_grid* g)
{
    if (!g) return 0;
    return g->L.dynamic_bytes + 256;
}

fdtd_status fdtd_save_state(fdtd_grid* g, void* dev_dst)
{
    if (!g || !dev_dst) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(g, "fdtd_save_state");
    if (dev_st != FDTD_OK) return dev_st;
    int64_t hdr[4] = {g->step, g->cur, 0x46445444, g->pe};
    char* D = static_cast<char*>(dev_dst);
    fdtd_status st = cuda_check(cudaMemcpyAsync(D, g->arena, g->L.dynamic_bytes, cudaMemcpyDeviceToDevice,
                                                g->stream), "save state");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(D + g->L.dynamic_bytes, hdr, sizeof(hdr), cudaMemcpyHostToDevice,
                                        g->stream), "save state");
    if (st != FDTD_OK) return st;
    return fdtd_sync(g);
}

fdtd_status fdtd_load_state(fdtd_grid* g, const void* dev_src)
{
    if (!g || !dev_src) return fail(FDTD_EINVAL, "null argument");
    const fdtd_status dev_st = check_device(g, "fdtd_load_state");
    if (dev_st != FDTD_OK) return dev_st;
    int64_t hdr[4];
    const char* S = static_cast<const char*>(dev_src);
    fdtd_status st = cuda_check(cudaMemcpyAsync(hdr, S + g->L.dynamic_bytes, sizeof(hdr), cudaMemcpyDeviceToHost,
                                                g->stream), "load state");
    if (st == FDTD_OK) st = fdtd_sync(g);
    if (st != FDTD_OK) return st;
    if (hdr[2] != 0x46445444 || (hdr[1] != 0 && hdr[1] != 1) || (hdr[3] != 0 && hdr[3] != 1))
        return fail(FDTD_EINVAL, "state blob does not come from fdtd_save_state");
    st = cuda_check(cudaMemcpyAsync(g->arena, S, g->L.dynamic_bytes, cudaMemcpyDeviceToDevice, g->stream),
                    "load state");
    if (st != FDTD_OK) return st;
    g->step = hdr[0];
    g->cur = int(hdr[1]);
    g->pe = int(hdr[3]);
    return fdtd_sync(g);
}

int64_t fdtd_get_step(const fdtd_grid* g) { return g ? g->step : -1; }

fdtd_status fdtd_set_step(fdtd_grid* g, int64_t n)
{
    if (!g || n < 0) return fail(FDTD_EINVAL, "invalid argument");
    g->step = n;
    return FDTD_OK;
}

double fdtd_get_dt(const fdtd_grid* g) { return g ? g->dt : 0.0; }

int64_t fdtd_antenna_points(const fdtd_grid* g, int component)
{
    if (!g || component < 0 || component > 5) return -1;
    return g->counts[component];
}

void fdtd_destroy_grid(fdtd_grid* g) { delete g; }

fdtd_status fdtd_set_tile(fdtd_grid* g, int variant, int ty, int lz)
{
    if (!g) return fail(FDTD_EINVAL, "null grid");
    if (variant < 0 || variant > 7) return fail(FDTD_EINVAL, "variant=%d not in {0, ..., 7}", variant);
    if (ty != 4 && ty != 8 && ty != 16) return fail(FDTD_EINVAL, "ty=%d not in {4, 8, 16}", ty);
    if (variant == 7 && (ty == 4 || g->desc.precision != FDTD_F32))
        return fail(FDTD_EINVAL, "variant 7 takes FP32 grids and ty 8 or 16");
    if (variant == 6 && g->desc.nz > 65535) return fail(FDTD_EINVAL, "variant 6 takes nz <= 65535");
    if (variant != 5 && needs_cell_passes(g))
        return fail(FDTD_EINVAL, "a grid with z walls or a wall source takes tile variant 5");
    if ((variant == 1 || variant == 2 || variant == 4) && ty == 16 && g->desc.precision == FDTD_F64)
        return fail(FDTD_EINVAL, "the TMA variants have no FP64 32x16 tile");
    if (lz < 1) return fail(FDTD_EINVAL, "lz=%d < 1", lz);
    g->tile.variant = variant;
    g->tile.tx = 32;
    g->tile.ty = ty;
    g->tile.lz = lz > g->desc.nz ? g->desc.nz : lz;
    return FDTD_OK;
}

fdtd_status fdtd_set_balance(fdtd_grid* g, float w_shell, float w_antenna)
{
    if (!g) return fail(FDTD_EINVAL, "null grid");
    if (!(w_shell >= 0.0f && w_shell <= 16.0f) || !(w_antenna >= 0.0f && w_antenna <= 16.0f))
        return fail(FDTD_EINVAL, "balance weights %g, %g outside [0, 16]", w_shell, w_antenna);
    g->tile.w_shell = w_shell;
    g->tile.w_ant = w_antenna;
    g->tile.measured = false;
    return FDTD_OK;
}

fdtd_status fdtd_get_balance(const fdtd_grid* g, float* w_shell, float* w_antenna)
{
    if (!g || !w_shell || !w_antenna) return fail(FDTD_EINVAL, "null argument");
    *w_shell = g->tile.measured ? -1.0f : g->tile.w_shell;
    *w_antenna = g->tile.measured ? -1.0f : g->tile.w_ant;
    return FDTD_OK;
}

fdtd_status fdtd_get_tile(const fdtd_grid* g, int* variant, int* ty, int* lz)
{
    if (!g || !variant || !ty || !lz) return fail(FDTD_EINVAL, "null argument");
    *variant = g->tile.variant;
    *ty = g->tile.ty;
    *lz = g->tile.lz;
    return FDTD_OK;
}

// Time every (ty, lz) candidate on this grid with CUDA events and keep the
// fastest.  The state is saved to `scratch_state` (fdtd_state_bytes bytes of
// device memory owned by the caller) first and restored afterwards.
fdtd_status fdtd_autotune(fdtd_grid* g, int steps, void* scratch_state)
{
    if (!g || !scratch_state || steps < 1) return fail(FDTD_EINVAL, "invalid argument");
    const fdtd_status dev_st = check_device(g, "fdtd_autotune");
    if (dev_st != FDTD_OK) return dev_st;
    if (g->batch_refs > 0) return not_batched(g, "fdtd_autotune");
    g->fault = 0;
    fdtd_status st = fdtd_save_state(g, scratch_state);
    if (st != FDTD_OK) return st;
    struct Cand { int variant, ty; float w_shell = 0.0f, w_ant = 0.0f; };
    std::vector<Cand> cands = {{6, 4}, {6, 8}, {6, 16}, {5, 4}, {5, 8}, {5, 16}, {4, 4}, {4, 8}, {4, 16}, {3, 4},
                               {3, 8}, {3, 16}, {2, 8}, {2, 16}, {1, 4}, {1, 8}, {1, 16}, {0, 4}, {0, 8}, {0, 16}};
    if (g->desc.precision == FDTD_F64)
        cands = {{6, 4}, {6, 8}, {6, 16}, {5, 4}, {5, 8}, {5, 16}, {4, 4}, {4, 8}, {3, 4}, {3, 8}, {2, 8}, {2, 4},
                 {1, 4}, {1, 8}, {0, 4}, {0, 8}};
    if (g->desc.nz > 65535) cands.erase(cands.begin(), cands.begin() + 3);   // variant 6 takes nz <= 65535
    if (g->desc.precision == FDTD_F32)   // variant 7 with its work-split weights (shell, antenna)
        cands.insert(cands.begin(), {{7, 16, 0.0f, 0.0f}, {7, 16, 0.15f, 0.1f}, {7, 16, 0.3f, 0.2f},
                                     {7, 16, 0.45f, 0.3f}, {7, 16, 0.3f, 0.4f}, {7, 16, 0.6f, 0.4f},
                                     {7, 8, 0.3f, 0.2f}});
    if (needs_cell_passes(g)) cands = {{5, 4}, {5, 8}, {5, 16}};
    const int nz = g->desc.nz;
    std::vector<int> lzs;
    for (int segs : {1, 2, 3, 4, 6, 8, 12, 16}) {
        int lz = (nz + segs - 1) / segs;
        if (lz >= 4 || segs == 1) {
            bool dup = false;
            for (int v : lzs) dup |= (v == lz);
            if (!dup) lzs.push_back(lz);
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(FDTD_ECUDA, "event create failed");
    // every candidate runs the same even number of steps (variant 7 steps in pairs)
    const int nrun = steps + (steps & 1);
    float best = 1e30f;
    TileConfig best_tc = g->tile;
    cudaError_t err = cudaSuccess;
    for (const Cand& cd : cands)
        for (int lz : lzs) {
            if (cd.variant >= 5 && lz != lzs[0]) continue;   // one cell per thread: no z segments
            TileConfig tc; tc.variant = cd.variant; tc.tx = 32; tc.ty = cd.ty; tc.lz = lz;
            if (cd.variant == 7) { tc.w_shell = cd.w_shell; tc.w_ant = cd.w_ant; tc.lz = 1; }
            err = run_steps(g, 2, tc);   // warm-up
            if (err != cudaSuccess) break;
            cudaEventRecord(e0, g->stream);
            err = run_steps(g, nrun, tc);
            cudaEventRecord(e1, g->stream);
            if (err != cudaSuccess) break;
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; best_tc = tc; }
        }
    // variant 7: the fastest weights' ranges refined on measured CTA times,
    // with the windows row by row and with the rows interleaved; keep the
    // fastest
    const TileConfig weights_tc = best_tc;
    for (int order = 1; order <= 2 && err == cudaSuccess && weights_tc.variant == 7; ++order) {
        TileConfig tc = weights_tc;
        tc.lz = order;
        err = tb2_measure(g, tc);
        if (err != cudaSuccess) break;
        tc.measured = true;
        err = run_steps(g, 2, tc);   // warm-up
        if (err != cudaSuccess) break;
        cudaEventRecord(e0, g->stream);
        err = run_steps(g, nrun, tc);
        cudaEventRecord(e1, g->stream);
        if (err != cudaSuccess) break;
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_tc = tc; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->fault = 0;
    st = fdtd_load_state(g, scratch_state);
    if (err != cudaSuccess) return cuda_check(err, "autotune");
    g->tile = best_tc;
    return st;
}

fdtd_status fdtd_source_coefficients(const fdtd_grid_desc* d, const fdtd_annulus_desc* s, double* out,
                                     uint8_t* out_mask)
{
    fdtd_status st = validate(d);
    if (st != FDTD_OK) return st;
    if (!s || !out || !out_mask) return fail(FDTD_EINVAL, "null argument");
    st = validate_source(*d, s);
    if (st != FDTD_OK) return st;
    GridSpec gs{d->nx, d->ny, d->nz, d->npml, d->dx, d->dy, d->dz, grid_dt(*d)};
    SourceSpec ss{s->m, s->theta, s->pol, s->mode, s->E0, s->r_center, s->thickness, s->inject};
    std::vector<std::complex<double>> coef;
    std::vector<uint8_t> mask;
    int64_t counts[6];
    source_tables(gs, ss, nullptr, nullptr, coef, mask, counts);
    std::memcpy(out, coef.data(), coef.size() * 16);
    std::memcpy(out_mask, mask.data(), mask.size());
    return FDTD_OK;
}

double fdtd_bessel_j(int n, double x) { return bessel_j(n, x); }

const char* fdtd_status_string(fdtd_status s)
{
    switch (s) {
        case FDTD_OK: return "ok";
        case FDTD_EINVAL: return "invalid argument";
        case FDTD_ENOMEM: return "out of memory";
        case FDTD_ECUDA: return "CUDA error";
        case FDTD_ETIMEOUT: return "device wait timed out";
        case FDTD_ESTATE: return "invalid state";
    }
    return "unknown status";
}

const char* fdtd_last_error(void) { return g_last_error; }

}  // extern "C"
