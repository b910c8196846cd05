// split.cu -- launches of the two-pass Yee steps: yee_h_pass + yee_e_pass
// (plain loads, fluence in the E pass) and yee_hflu_tma + yee_e_pass
// (TMA-staged H pass with the fluence term, plain-load E pass).
#include <cuda_runtime.h>

#include "grid_impl.h"
#include "tma_host.h"
#include "yee_cell.cuh"
#include "yee_step_cell.cuh"
#include "yee_hflu_tma.cuh"
#include "yee_split.cuh"

namespace fdtd {

// Tensor maps of yee_hflu_tma: E^n and H^{n-1/2} of copy `cur` in boxes of
// HFluTile::BX x (TY+1) at (i0, j0), the fluence in 32 x TY boxes.
template <typename real, int TY>
inline bool hflu_maps(fdtd_grid* g, int cur, TmaMaps** out)
{
    int sl = ty_slot(TY);
    if (!g->hmaps_ok[cur][sl]) {
        using T = HFluTile<real, TY>;
        char* A = static_cast<char*>(g->arena);
        TmaMaps& m = g->hmaps[cur][sl];
        bool ok = true;
        for (int c = 0; c < 3; ++c) {
            ok = ok && encode_map(&m.e[c], A + g->L.field[cur][c], sizeof(real), g->desc, g->L.pitch, T::BX, T::BY);
            ok = ok && encode_map(&m.h[c], A + g->L.field[cur][3 + c], sizeof(real), g->desc, g->L.pitch, T::BX,
                                  T::BY);
        }
        void* fbase = g->desc.fluence ? static_cast<void*>(A + g->L.fluence) : static_cast<void*>(A + g->L.field[cur][0]);
        ok = ok && encode_map(&m.f, fbase, 8, g->desc, g->L.pitch, T::FBX, T::FBY);
        if (!ok) return false;
        g->hmaps_ok[cur][sl] = true;
    }
    *out = &g->hmaps[cur][sl];
    return true;
}

// Two passes (H, then E with the fluence term), 32 x TY threads, one column each.
template <typename real, int TY>
static cudaError_t launch_split(const fdtd_grid* g, int cur, long long n, int lz, cudaStream_t s, cudaEvent_t mid)
{
    dim3 block(32, TY);
    dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TY - 1) / TY, (g->desc.nz + lz - 1) / lz);
    const size_t smem = size_t(lz) * 2 * sizeof(real);
    static size_t attr_set = 0;
    if (smem > 48 * 1024 && smem > attr_set) {
        cudaError_t e = cudaFuncSetAttribute(yee_h_pass<real, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(yee_e_pass<real, TY, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem));
        if (e != cudaSuccess) return e;
        attr_set = smem;
    }
    const StepArgs<real> a = make_args<real>(g, cur);
    yee_h_pass<real, TY><<<grid, block, smem, s>>>(a, n, lz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mid) cudaEventRecord(mid, s);
    yee_e_pass<real, TY, true><<<grid, block, smem, s>>>(a, n, lz);
    return cudaGetLastError();
}

// TMA-staged H pass with the fluence term (S stages), then the E pass.
template <typename real, int TY, int S>
static cudaError_t launch_hflu(const fdtd_grid* cg, int cur, long long n, int lz, cudaStream_t s, cudaEvent_t mid)
{
    fdtd_grid* g = const_cast<fdtd_grid*>(cg);
    using T = HFluTile<real, TY>;
    const size_t smem = T::smem_bytes(S, lz);
    const size_t esmem = size_t(lz) * 2 * sizeof(real);
    static size_t attr_set = 0, eattr_set = 0;
    if (smem > attr_set) {
        cudaError_t e = cudaFuncSetAttribute(yee_hflu_tma<real, TY, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(smem));
        if (e != cudaSuccess) return e;
        attr_set = smem;
    }
    if (esmem > 48 * 1024 && esmem > eattr_set) {
        cudaError_t e = cudaFuncSetAttribute(yee_e_pass<real, TY, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(esmem));
        if (e != cudaSuccess) return e;
        eattr_set = esmem;
    }
    TmaMaps* m = nullptr;
    if (!hflu_maps<real, TY>(g, cur, &m)) return cudaErrorInvalidValue;
    dim3 block(32, TY);
    dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TY - 1) / TY, (g->desc.nz + lz - 1) / lz);
    int* err = reinterpret_cast<int*>(static_cast<char*>(g->arena) + g->L.err);
    const StepArgs<real> a = make_args<real>(g, cur);
    yee_hflu_tma<real, TY, S><<<grid, block, smem, s>>>(a, *m, n, lz, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (mid) cudaEventRecord(mid, s);
    yee_e_pass<real, TY, false><<<grid, block, esmem, s>>>(a, n, lz);
    return cudaGetLastError();
}

// One cell-parallel pass: yee_step_cell, 32 x TY threads, one cell each.
template <typename real, int TY>
static cudaError_t launch_step_cell(const fdtd_grid* g, int cur, long long n, cudaStream_t s)
{
    if (g->desc.nz > 65535) return cudaErrorInvalidConfiguration;
    const StepTime<real> t = step_time<real>(g->srct, nullptr, g->dt, n);
    dim3 block(32, TY);
    dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TY - 1) / TY, g->desc.nz);
    yee_step_cell<real, TY><<<grid, block, 0, s>>>(make_args<real>(g, cur), t);
    return cudaGetLastError();
}

// FP64 grids with an antenna (z-periodic, no wall sheet) add its source in
// antenna_add after each pass instead of inside it.
template <typename real>
static cudaError_t antenna_pass(const fdtd_grid* g, const StepArgs<real>& a, int side, Cpx<real> t, cudaStream_t s)
{
    const int ncols = g->ant_cols[side];
    if (ncols == 0) return cudaSuccess;
    const int* cols = reinterpret_cast<const int*>(static_cast<const char*>(g->arena) + g->L.alist) +
                      (side == 0 ? 0 : g->ant_cols[0]);
    const long long pts = (long long)ncols * g->desc.nz;
    const unsigned blocks = unsigned((pts + 255) / 256);
    if (side == 0)
        antenna_add<real><<<blocks, 256, 0, s>>>(a, cols, ncols, 3, t, a.hout[0], a.hout[1], a.hout[2]);
    else
        antenna_add<real><<<blocks, 256, 0, s>>>(a, cols, ncols, 0, t, a.eout[0], a.eout[1], a.eout[2]);
    return cudaGetLastError();
}

// Cell-parallel passes: yee_h_cell then yee_e_cell (with the fluence term),
// or yee_h_cell_w then yee_e_cell_w on grids with z walls or a wall sheet
// (FP64 z-periodic grids: each pass followed by antenna_add);
// 32 x TY threads, one cell each, one plane per grid z index.  Grids of more
// than kMaxPlanes planes launch each pass in chunks of planes (the H pass's
// chunks in order, the E pass's in reverse, as its blocks run).
constexpr int kMaxPlanes = 65535;   // gridDim.z limit
template <typename real, int TY>
static cudaError_t launch_cell(const fdtd_grid* g, int cur, long long n, cudaStream_t s, cudaEvent_t mid)
{
    const StepTime<real> t = step_time<real>(g->srct, g->has_wall ? &g->wallt : nullptr, g->dt, n);
    const int nz = g->desc.nz, nchunk = (nz + kMaxPlanes - 1) / kMaxPlanes;
    dim3 block(32, TY);
    const bool wall = needs_cell_passes(g);   // z walls or a wall sheet: the *_w kernels
    const bool apart = sizeof(real) == 8 && g->has_source && g->ant_apart && !wall;
    const StepArgs<real> full = make_args<real>(g, cur);
    StepArgs<real> a = full;
    if (apart) a.smask = nullptr;   // the passes run without the antenna
    for (int c = 0; c < nchunk; ++c) {
        a.kbase = c * kMaxPlanes;
        dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TY - 1) / TY, nz - a.kbase < kMaxPlanes ? nz - a.kbase : kMaxPlanes);
        if (wall) yee_h_cell_w<real, TY><<<grid, block, 0, s>>>(a, t);
        else yee_h_cell<real, TY><<<grid, block, 0, s>>>(a, t);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (apart) {
        const cudaError_t e = antenna_pass<real>(g, full, 0, t.th, s);
        if (e != cudaSuccess) return e;
    }
    if (mid) cudaEventRecord(mid, s);
    for (int c = nchunk - 1; c >= 0; --c) {
        a.kbase = c * kMaxPlanes;
        dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TY - 1) / TY, nz - a.kbase < kMaxPlanes ? nz - a.kbase : kMaxPlanes);
        if (wall) yee_e_cell_w<real, TY><<<grid, block, 0, s>>>(a, t);
        else yee_e_cell<real, TY><<<grid, block, 0, s>>>(a, t);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (apart) return antenna_pass<real>(g, full, 1, t.te, s);
    return cudaSuccess;
}

cudaError_t launch_split(const fdtd_grid* g, int cur, long long n, const TileConfig& tc, cudaStream_t s,
                         cudaEvent_t mid)
{
    const bool f32 = g->desc.precision == FDTD_F32;
    if (tc.variant == 6) {
        switch (tc.ty) {
            case 4: return f32 ? launch_step_cell<float, 4>(g, cur, n, s) : launch_step_cell<double, 4>(g, cur, n, s);
            case 16:
                return f32 ? launch_step_cell<float, 16>(g, cur, n, s) : launch_step_cell<double, 16>(g, cur, n, s);
            default: return f32 ? launch_step_cell<float, 8>(g, cur, n, s) : launch_step_cell<double, 8>(g, cur, n, s);
        }
    }
    if (tc.variant == 5) {
        switch (tc.ty) {
            case 4: return f32 ? launch_cell<float, 4>(g, cur, n, s, mid) : launch_cell<double, 4>(g, cur, n, s, mid);
            case 16: return f32 ? launch_cell<float, 16>(g, cur, n, s, mid) : launch_cell<double, 16>(g, cur, n, s, mid);
            default: return f32 ? launch_cell<float, 8>(g, cur, n, s, mid) : launch_cell<double, 8>(g, cur, n, s, mid);
        }
    }
    if (tc.variant == 4) {
        if (f32) {
            switch (tc.ty) {
                case 4: return launch_hflu<float, 4, 6>(g, cur, n, tc.lz, s, mid);
                case 16: return launch_hflu<float, 16, 4>(g, cur, n, tc.lz, s, mid);
                default: return launch_hflu<float, 8, 4>(g, cur, n, tc.lz, s, mid);
            }
        }
        return tc.ty == 4 ? launch_hflu<double, 4, 5>(g, cur, n, tc.lz, s, mid) : launch_hflu<double, 8, 4>(g, cur, n, tc.lz, s, mid);
    }
    switch (tc.ty) {
        case 4: return f32 ? launch_split<float, 4>(g, cur, n, tc.lz, s, mid) : launch_split<double, 4>(g, cur, n, tc.lz, s, mid);
        case 16:
            return f32 ? launch_split<float, 16>(g, cur, n, tc.lz, s, mid) : launch_split<double, 16>(g, cur, n, tc.lz, s, mid);
        default: return f32 ? launch_split<float, 8>(g, cur, n, tc.lz, s, mid) : launch_split<double, 8>(g, cur, n, tc.lz, s, mid);
    }
}

}  // namespace fdtd
