// grid_impl.h -- host-side grid object and arena layout (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/fdtd.h"
#include "yee_fused.cuh"
#include "yee_tma.cuh"
#include "yee_cell.cuh"

namespace fdtd {

struct Layout {
    size_t elem = 4;
    int pitch = 0;
    size_t field_elems = 0, psx_elems = 0, psy_elems = 0;
    size_t field[2][6] = {};
    size_t phx[2][2] = {}, phy[2][2] = {};
    size_t pex[2][2] = {}, pey[2][2] = {};   // [copy][component]: E psi, updated in place except by variant 7
    size_t psz_elems = 0;                 // z shell psi of z-walled grids: [2 npml_z][ny][pitch]
    size_t phz[2][2] = {}, pez[2] = {};   // Hxz, Hyz (ping-pong); Exz, Eyz (in place)
    size_t fluence = 0;
    size_t dynamic_bytes = 0;
    size_t chx = 0, cex = 0, chy = 0, cey = 0, chz = 0, cez = 0;
    size_t prof[12] = {};  // bhx ahx bex aex bhy ahy bey aey bhz ahz bez aez
    size_t wcoef = 0, wcoef32 = 0;   // wall-source column coefficients (FP64, FP32)
    size_t smask = 0, scoef = 0, scoef32 = 0, zph = 0, zph32 = 0;
    size_t scoef_unw = 0, wamp = 0, wphase = 0;   // unweighted coefficients and the weights
    size_t flu_out = 0;    // dense FP64 export of the fluence
    size_t tb2prof = 0;    // variant 7: per-CTA cycle counters of a measuring launch
    size_t alist = 0;      // antenna columns (int): those with H points, then those with E points
    size_t err = 0;        // device error word (int)
    size_t total = 0;
};

// variant 0: plain loads into a shared-memory ring (yee_step_fused);
// variant 1: TMA-staged planes with mbarriers (yee_step_tma), one row per thread;
// variant 2: the same with two rows of the tile per thread;
// variant 3: two plain-load passes, H then E with the fluence term;
// variant 4: two passes, TMA-staged H with the fluence term, then plain-load E;
// variant 5: two cell-parallel passes, H then E with the fluence term;
// variant 6: one cell-parallel pass, neighbour H recomputed in registers;
// variant 7: two steps per launch (temporal blocking, yee_tb2), FP32,
//            windows of 32 x ty columns (ty = 8 or 16); an odd step count
//            ends with one step of variant 5.
struct TileConfig {
    int variant = 1, tx = 32, ty = 8, lz = 32;
    // variant 7: extra cost per plane of a window holding CPML shell / antenna
    // columns, relative to a plain window (the CTAs' work ranges are balanced
    // on these estimates)
    float w_shell = 0.25f, w_ant = 0.2f;
    // variant 7: run the ranges refined from measured per-CTA times
    // (fdtd_grid::tb2_refined) instead of those of the weights above
    bool measured = false;
};

fdtd_status fail(fdtd_status st, const char* fmt, ...);
fdtd_status cuda_check(cudaError_t e, const char* what);
bool compute_layout(const fdtd_grid_desc& d, Layout& L);
fdtd_status validate(const fdtd_grid_desc* d);
// EINVAL unless the current CUDA device is the one the grid was created on
// (every entry point that queues work for a grid or reads its memory checks
// this first: the grid's arena and stream belong to that device).
fdtd_status check_device(const fdtd_grid* g, const char* what);
// Looks up (again) the device address of the no-allocation read-out's fixed
// staging array on the current device.  Called by fdtd_create_grid, where
// allocating is allowed: the lookup loads the array's module on that device.
fdtd_status noalloc_prepare(int device);
double grid_dt(const fdtd_grid_desc& d);
TileConfig default_tile(const fdtd_grid_desc& d, int sm_count);

}  // namespace fdtd

struct fdtd_grid {
    fdtd_grid_desc desc;
    fdtd::Layout L;
    void* arena;
    size_t arena_bytes;
    cudaStream_t stream;
    double dt;
    int64_t step;
    int cur;                 // which ping-pong copy holds the current state
    int pe;                  // which copy of the E-side psi is current (flipped by variant 7)
    bool has_source;
    fdtd_annulus_desc src;
    fdtd::SrcTime srct;
    int64_t counts[6];
    int sm_count;
    int device;                 // CUDA device current at fdtd_create_grid
    fdtd::TileConfig tile;
    fdtd::TmaMaps maps[2][3];   // [read copy][ty = 4, 8, 16]
    bool maps_ok[2][3];
    fdtd::TmaMaps hmaps[2][3];  // the same for the boxes of yee_hflu_tma
    bool hmaps_ok[2][3];
    int fault;                  // fdtd_debug_inject_fault: applies to the next step only
    int batch_refs;             // batches holding this grid (their kernels hold copies of its arguments)
    bool has_wall;              // fdtd_set_wall_source
    fdtd_wall_desc wall;
    fdtd::SrcTime wallt;        // time envelope of the wall source
    std::vector<uint8_t> hmask; // antenna component mask per (i, j) column (host copy), empty without a source
    int src_gen;                // bumped whenever the antenna's columns (hmask) change
    int ant_cols[2];            // antenna columns with H points, with E points (lists at L.alist)
    bool ant_apart;             // the FP64 cell passes may add the source in antenna_add (no antenna
                                // column on the i = 0 or j = 0 wall, where the E pass zeroes after it)
    std::vector<long long> tb2_start;   // variant 7: cached CTA work ranges
    struct {
        int ry, slots, src_gen, cost_gen, order;
        float w_shell, w_ant;
        bool measured;
    } tb2_key;                          // what they were computed for (ry 0: nothing cached)
    std::vector<long long> tb2_refined; // variant 7: CTA ranges refined from measured per-CTA times
    int tb2_ref_ry, tb2_ref_slots;      // the window height and CTA count they are for (ry 0: none)
    int tb2_ref_src;                    // the antenna generation they were measured with
    int tb2_ref_order;                  // the window order they were refined for
    int tb2_ref_gen;                    // bumped whenever tb2_refined changes
    bool tb2_profile;                   // the next variant-7 launches record per-CTA cycles
};

namespace fdtd {
template <typename real>
StepArgs<real> make_args(const fdtd_grid* g, int cur);
// One step on stream s.  `mid`, if not null, is recorded between the two
// kernels of a two-pass variant (ignored by the one-pass variants).
cudaError_t launch_step(const fdtd_grid* g, int cur, long long n, const TileConfig& tc, cudaStream_t s,
                        cudaEvent_t mid = nullptr);
// True if the grid needs the cell passes of tile variant 5 (z walls or a
// wall source: the other variants implement z-periodic grids only).
inline bool needs_cell_passes(const fdtd_grid* g)
{
    return g->desc.z_boundary == FDTD_Z_WALLS || g->has_wall;
}
// Kernel launches per step of a tile configuration (1 or 2; variant 7 launches
// once per two steps).
inline int passes_per_step(const TileConfig& tc) { return tc.variant >= 3 && tc.variant <= 5 ? 2 : 1; }
// Tile variant 7: two steps n, n+1 from copy `cur` (fields, H psi) and E psi
// copy g->pe into the other copies.  FP32, z-periodic grids without a wall
// source only.
cudaError_t launch_tb2(const fdtd_grid* g, int cur, long long n, const TileConfig& tc, cudaStream_t s);
// Windows of variant 7 with 32 x ry columns on grid d: t along x, u along y.
void tb2_windows(const fdtd_grid_desc& d, int ry, int* t, int* u);
// Moves the boundaries of the cached ranges (windows of 32 x ry columns,
// `slots` CTAs) `step` (in (0, 1]) of the way to where the CTAs' times, from
// the SM cycles each took in the measured launches (cycles[c]) spread evenly
// over its items, become equal; stored on the grid for the plans of
// tc.measured.
void tb2_refine(fdtd_grid* g, int ry, int slots, const unsigned long long* cycles, double step);
// The arithmetic of tb2_refine: new range starts from the starts s (slots + 1)
// and the CTAs' cycles.
std::vector<long long> tb2_refined_ranges(const std::vector<long long>& s, const unsigned long long* cycles,
                                          double step);
// CTAs of one variant-7 launch on grid g with windows of 32 x ry columns.
int tb2_slots(const fdtd_grid* g, int ry);
// The same two steps with their time factors from a device table of
// StepTime<float> (entries i0, i1), on at most max_ctas CTAs (a batch runs
// several grids side by side): the batched graph's launch.
cudaError_t launch_tb2_table(const fdtd_grid* g, int cur, const StepTime<float>* times, int i0, int i1,
                             int max_ctas, cudaStream_t s);
// The tile of the single step that completes an odd step count of variant 7.
inline TileConfig single_step_tile(const TileConfig& tc)
{
    if (tc.variant != 7) return tc;
    TileConfig one;
    one.variant = 5; one.tx = 32; one.ty = 4; one.lz = tc.lz;
    return one;
}
// The cell-parallel and two-pass steps on stream s: variant 3 yee_h_pass then
// yee_e_pass (with the fluence term); variant 4 yee_hflu_tma (with the
// fluence term) then yee_e_pass; variant 5 yee_h_cell then yee_e_cell;
// variant 6 yee_step_cell.
cudaError_t launch_split(const fdtd_grid* g, int cur, long long n, const TileConfig& tc, cudaStream_t s,
                         cudaEvent_t mid);
}  // namespace fdtd
