// batch.cu -- many independent Bessel-antenna grids (different orders, cone
// angles, ring radii and transverse sizes) advanced together.
//
// Each grid runs the unchanged method of its own descriptor (Section 4,
// Eq. 12-13).  A CUDA graph holds K = 64 consecutive steps of every grid;
// one replay (or, for the persistent cell engine, one cooperative launch per
// group of grids) advances them all by K steps.  Three engines:
//   * persistent (FDTD_BATCH_PERSISTENT): the batch flattens every grid's
//     (32 x TR tile, z segment) blocks into one work list; one persistent
//     kernel launch per step, one CTA per resident slot (SM count x
//     occupancy), walks the list with a grid stride and marches each block
//     with the TMA-staged one-pass step (tma_march).  The CTA's mbarriers are
//     initialised once and their phases carried from block to block; a
//     one-thread kernel at the end of the graph advances the device step
//     counter from which the source phases are taken.
//   * persistent cell passes (FDTD_BATCH_PERSISTENT_CELL): one cooperative
//     kernel launch runs up to K steps of every grid.  The 32 x 4 cell
//     blocks of all grids form one list; the CTAs (one per resident slot)
//     take runs of kPCellChunk consecutive blocks, in order, from a per-pass
//     counter (the E pass from the end of the list), then single blocks near
//     the end of the pass, so that the blocks in flight stay a narrow front
//     whose neighbours are in L2, as under the hardware block scheduler, and
//     a pass ends within about one block of its average.  H pass of every grid, grid barrier, E pass, barrier, and so
//     on.  The cell arithmetic is that of tile variant 5, bit for bit; the
//     barriers are bounded waits.
//   * cell passes (FDTD_BATCH_CELL, the default): each grid steps with the
//     cell-parallel H and E passes of the single-grid variant 5 (32 x 4 x 1
//     blocks, one thread per cell).  The graph gives every grid its own
//     branch (up to kCellBranches concurrent streams, shared round-robin), so
//     the passes of small grids run side by side instead of each leaving the
//     GPU idle in its tail.  The per-step source time factors of every grid
//     are evaluated on the host in FP64, as for a single grid, and copied
//     into a device table ahead of each replay; the kernels read their step's
//     entry.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "grid_impl.h"
#include "tma_host.h"
#include "yee_cell.cuh"
#include "yee_tma.cuh"

namespace fdtd {

struct BatchHeader {
    int ngrids, nitems;
    long long counter;   // steps taken by the batch since creation
    int err;             // device error word
    int fault;           // test hook: 1 = CTA 0 of the next persistent cell launch never arrives
};

template <typename real>
struct alignas(128) BatchGrid {
    TmaMaps maps[2];        // by copy being read
    StepArgs<real> args[2];
    long long step0;        // the grid's step counter when the batch was created
    int item0, ntx, nty, nseg, lz;
};

constexpr int kBatchLz = 32;   // z segment of a batched block

// One CTA of 32 x (TR / R) threads per resident slot; each block is a
// 32 x TR tile of one grid.
template <typename real, int TR, int R, int S>
__global__ void __launch_bounds__(32 * (TR / R), MinCtas<real, TR, R>::value)
yee_batch_tma(BatchHeader* __restrict__ hdr, const BatchGrid<real>* __restrict__ grids, int parity, int offset)
{
    constexpr int NT = 32 * (TR / R);
    const MarchSmem<real, TR, S> sm = march_smem_init<real, TR, S>(kBatchLz);
    __shared__ __align__(16) unsigned char sargs_raw[sizeof(StepArgs<real>)];
    const StepArgs<real>& sa = *reinterpret_cast<const StepArgs<real>*>(sargs_raw);
    const int ngrids = hdr->ngrids, nitems = hdr->nitems;
    const long long done = hdr->counter;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    int gq = 0;
    #pragma unroll 1
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        int g = 0;
        while (g + 1 < ngrids && grids[g + 1].item0 <= item) ++g;
        const BatchGrid<real>& G = grids[g];
        __syncthreads();   // every reader of the previous block's arguments is done
        const int* src = reinterpret_cast<const int*>(&G.args[parity]);
        int* dst = reinterpret_cast<int*>(sargs_raw);
        for (int w = tid; w < int(sizeof(StepArgs<real>) / 4); w += NT) dst[w] = src[w];
        __syncthreads();   // publish the copied arguments before tma_march reads them
        int local = item - G.item0;
        const int bz = local % G.nseg;
        local /= G.nseg;
        const int bx = local % G.ntx, by = local / G.ntx;
        const int kb = bz * G.lz;
        const int nz = G.args[parity].nz;
        gq = tma_march_any<real, TR, R, S>(sa, G.maps[parity], G.step0 + done + offset, bx * 32, by * TR, kb,
                                           min(kb + G.lz, nz), &hdr->err, sm, gq);
        if (gq < 0) return;
    }
}

__global__ void batch_advance(BatchHeader* hdr, int k)
{
    hdr->counter += k;
}

constexpr int kBatchGraphSteps = 64;   // even, so a replay leaves the read copy unchanged

// ---- cell-pass engine
constexpr int kCellTY = 4;          // 32 x 4 x 1 cell blocks (tile variant 5)
constexpr int kCellBranches = 16;   // concurrent graph branches (grids share them round-robin)

// ---- persistent cell engine
// Kernel parameter of one persistent cell launch: a group of at most
// kPCellGroup grids.  Passed as a __grid_constant__ parameter, so that the
// cell code reads each grid's arguments from the constant bank with a
// uniform runtime index, as the single-grid kernels read theirs.
constexpr int kPCellGroup = 24;
constexpr int kPCellChunk = 4;   // consecutive blocks per counter ticket
template <typename real>
struct PCellParams {
    StepArgs<real> args[kPCellGroup][2];   // [grid][copy being read]
    int ntx[kPCellGroup], nty[kPCellGroup], nz[kPCellGroup];   // 32 x 4 blocks along x, y; planes
    int block0[kPCellGroup + 1];              // first block of each grid; block0[ngrids] = nblocks
    int wall[kPCellGroup];                    // z walls or a wall sheet: the wall code path
    int ngrids, nblocks;
    int q0, nall;                             // the group's first grid in the batch; grids in the batch
    int nsteps, parity0;
    BatchHeader* hdr;
    const StepTime<real>* times;              // [step][batch grid]
    unsigned* bar;                            // barrier words (kBarBytes, layout at grid_barrier)
};
// kernel parameters may take 32764 bytes (sm_70 and later, CUDA 12.1 and later)
static_assert(sizeof(PCellParams<float>) <= 32764 && sizeof(PCellParams<double>) <= 32764,
              "a group's arguments must fit in one kernel parameter");

// Barrier words of the persistent cell engine, one 128-byte line each:
// [0] arrivals of group leaders, [32] generation, [64 + 32 pass] block
// counter of each pass, [128 + 32 g] arrivals within group g of kBarGroup CTAs.
constexpr int kBarGroup = 32;
constexpr int kBarLine = 32;
constexpr size_t kBarBytes = 32768;   // room for 4864 CTAs (32 per SM x 152 SMs)

// Grid-wide barrier of a cooperative launch (every CTA resident), in two
// levels so that no counter takes more than about kBarGroup arrivals: thread 0
// of each CTA arrives on its group's counter; the last of a group resets it
// and arrives on the leaders' counter; the last leader resets that and the
// block counter of the pass just finished (every CTA has stopped taking
// blocks from it), then advances the generation.  The others wait for the
// generation to move, for at most 2^32 SM cycles, or until another CTA has
// raised the error word.  Release / acquire fences on every arrival and
// after the wait make the field writes of the pass before visible to the
// loads of the pass after.  Returns false (error word set) if the wait gave
// up.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int pass, unsigned nblocks, int* err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int ok = 1;
        volatile unsigned* vgen = bar + kBarLine;
        volatile int* verr = err;
        const unsigned g0 = *vgen;
        const unsigned grp = blockIdx.x / kBarGroup;
        const unsigned gsize = nblocks - grp * kBarGroup < unsigned(kBarGroup) ? nblocks - grp * kBarGroup : kBarGroup;
        const unsigned ngroups = (nblocks + kBarGroup - 1) / kBarGroup;
        unsigned* gcount = bar + 4 * kBarLine + grp * kBarLine;
        bool last = false;
        __threadfence();
        if (atomicAdd(gcount, 1u) == gsize - 1) {
            *reinterpret_cast<volatile unsigned*>(gcount) = 0u;
            __threadfence();
            last = atomicAdd(bar, 1u) == ngroups - 1;
        }
        if (last) {
            *reinterpret_cast<volatile unsigned*>(bar) = 0u;
            *reinterpret_cast<volatile unsigned*>(bar + (2 + pass) * kBarLine) = 0u;
            __threadfence();
            atomicAdd(bar + kBarLine, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g0) {
                if (*verr != 0) { ok = 0; break; }
                if (clock64() - t0 > (1LL << 32)) { atomicExch(err, 3); ok = 0; break; }
            }
        }
        __threadfence();
        if (*verr != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Resident CTAs per SM of the persistent cell kernel: 40 registers (FP32) or
// 64 (FP64), the budgets of the single-grid E pass.
template <typename real>
struct BatchCellOcc { static constexpr int value = sizeof(real) == 8 ? 8 : 12; };

// `P.nsteps` steps of every grid of the group.
template <typename real>
__global__ void __launch_bounds__(32 * kCellTY, BatchCellOcc<real>::value)
yee_batch_cell(const __grid_constant__ PCellParams<real> P)
{
    if (P.hdr->fault == 1 && blockIdx.x == 0) return;   // fdtd_batch_debug_inject_fault
    __shared__ int4 s_blk;   // first block of the next run: grid, bx, by, k (grid < 0: the pass is done)
    __shared__ int s_len;    // blocks in the run
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    const int nb = P.nblocks;
    // ticket t of the pass -> its first block (grid, bx, by, k) and run
    // length: runs of kPCellChunk blocks, then single blocks for the last
    // 2 x gridDim.x blocks so that the pass ends within one block of its
    // average; the E pass walks the list from its end
    const int tail = nb < 2 * int(gridDim.x) ? nb : 2 * int(gridDim.x);
    const int nrun = (nb - tail) / kPCellChunk, head = nrun * kPCellChunk;
    auto decode = [&](unsigned t, int pass) {
        const long long b0 = t < unsigned(nrun) ? (long long)t * kPCellChunk : head + ((long long)t - nrun);
        if (b0 >= nb) { s_blk = make_int4(-1, 0, 0, 0); s_len = 0; return; }
        const int len = t < unsigned(nrun) ? kPCellChunk : 1;
        const int b = pass == 0 ? int(b0) : nb - 1 - int(b0);
        int q = 0;
        while (P.block0[q + 1] <= b) ++q;
        const int ntx = P.ntx[q], per = ntx * P.nty[q];
        int local = b - P.block0[q];
        const int k = local / per;
        local -= k * per;
        const int by = local / ntx;
        s_blk = make_int4(q, local - by * ntx, by, k);
        s_len = len;
    };
    #pragma unroll 1
    for (int s = 0; s < P.nsteps; ++s) {
        const int parity = P.parity0 ^ (s & 1);
        #pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            unsigned* ctr = P.bar + (2 + pass) * kBarLine;
            if (lead) decode(atomicAdd(ctr, 1u), pass);
            __syncthreads();
            int4 cur = s_blk;
            int len = s_len;
            #pragma unroll 1
            while (cur.x >= 0) {
                __syncthreads();   // every thread has read s_blk, s_len
                unsigned t_next = 0;
                if (lead) t_next = atomicAdd(ctr, 1u);   // fetched while this run is processed
                int q = cur.x, bx = cur.y, by = cur.z, k = cur.w;
                int ntx = P.ntx[q], nty = P.nty[q];
                #pragma unroll 1
                for (int n = len; n > 0; --n) {
                    const StepArgs<real>& sa = P.args[q][parity];
                    const StepTime<real>& T = P.times[s * P.nall + P.q0 + q];
                    const int i0 = bx * 32, j0 = by * kCellTY;
                    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
                    if (pass == 0) {
                        if (P.wall[q]) {
                            if (cell_gen_h<real, kCellTY>(sa, i0, j0) || cell_gen_z(sa, k))
                                h_cell<real, true, true, false>(sa, T.th, i, j, k);
                            else h_cell<real, false, true, false>(sa, T.th, i, j, k);
                        } else {
                            if (cell_gen_h<real, kCellTY>(sa, i0, j0)) h_cell<real, true, false, false>(sa, T.th, i, j, k);
                            else h_cell<real, false, false, false>(sa, T.th, i, j, k);
                        }
                        // next block of the list (the last one of a run moves nowhere)
                        if (n > 1 && ++bx == ntx) {
                            bx = 0;
                            if (++by == nty) {
                                by = 0;
                                if (++k == P.nz[q]) { k = 0; ++q; ntx = P.ntx[q]; nty = P.nty[q]; }
                            }
                        }
                    } else {
                        if (P.wall[q]) {
                            if (cell_gen_e<real, kCellTY>(sa, i0, j0) || cell_gen_z(sa, k))
                                e_cell<real, true, true, false>(sa, T.te, T.tw, i, j, k);
                            else e_cell<real, false, true, false>(sa, T.te, T.tw, i, j, k);
                        } else {
                            if (cell_gen_e<real, kCellTY>(sa, i0, j0)) e_cell<real, true, false, false>(sa, T.te, T.tw, i, j, k);
                            else e_cell<real, false, false, false>(sa, T.te, T.tw, i, j, k);
                        }
                        // previous block of the list
                        if (n > 1 && bx-- == 0) {
                            bx = ntx - 1;
                            if (by-- == 0) {
                                by = nty - 1;
                                if (k-- == 0) {
                                    --q;
                                    ntx = P.ntx[q]; nty = P.nty[q];
                                    k = P.nz[q] - 1; by = nty - 1; bx = ntx - 1;
                                }
                            }
                        }
                    }
                }
                if (lead) decode(t_next, pass);
                __syncthreads();
                cur = s_blk;
                len = s_len;
            }
            if (!grid_barrier(P.bar, pass, gridDim.x, &P.hdr->err)) return;
        }
    }
}

}  // namespace fdtd

using namespace fdtd;

struct fdtd_batch {
    std::vector<fdtd_grid*> grids;
    int precision;
    int engine;                      // FDTD_BATCH_PERSISTENT, _CELL or _PERSISTENT_CELL
    int ty, S;
    void* table;
    size_t table_bytes;
    size_t times_off;                // byte offset of the time table in `table`
    cudaStream_t stream;
    cudaStream_t capture;
    int nitems;                      // persistent TMA engine: work items
    int nblocks;                     // persistent TMA engine: resident CTAs
    int cell_blocks;                 // cell engines: blocks per step and pass
    std::vector<unsigned char> pc_params;   // persistent cell engine: PCellParams of each group
    std::vector<int> pc_blocks;             // resident CTAs of each group's launch
    size_t bar_off;                         // byte offset of its barrier words
    int fault;                       // fdtd_batch_debug_inject_fault pending
    cudaStream_t branch[kCellBranches];
    int nbranch;
    std::vector<unsigned char> host_times;
    int cur;
    int64_t step;
    cudaGraphExec_t exec[2][2];      // [engine][read copy at the replay's start]
    bool built[2][2];
};

namespace {

size_t grid_entry_bytes(int precision)
{
    return precision == FDTD_F64 ? sizeof(BatchGrid<double>) : sizeof(BatchGrid<float>);
}

size_t time_entry_bytes(int precision)
{
    return precision == FDTD_F64 ? sizeof(StepTime<double>) : sizeof(StepTime<float>);
}

// Table layout: header (256 B) | BatchGrid[n] | barrier words (kBarBytes) | time factors.
size_t bar_offset(int n, int precision)
{
    return (256 + grid_entry_bytes(precision) * size_t(n) + 255) / 256 * 256;
}

size_t times_offset(int n, int precision)
{
    return bar_offset(n, precision) + kBarBytes;
}

// ---- cell engine
void cell_fill(fdtd_batch* b)
{
    b->cell_blocks = 0;
    for (const fdtd_grid* g : b->grids)
        b->cell_blocks += ((g->desc.nx + 31) / 32) * ((g->desc.ny + kCellTY - 1) / kCellTY) * g->desc.nz;
}

// Step `step` of the replay for grid q on stream s (time factor times[step * n + q]).
template <typename real>
cudaError_t cell_launch_grid(fdtd_batch* b, int q, int parity, int step, cudaStream_t s)
{
    const fdtd_grid* g = b->grids[q];
    const StepTime<real>* times =
        reinterpret_cast<const StepTime<real>*>(static_cast<char*>(b->table) + b->times_off);
    const int index = step * int(b->grids.size()) + q;
    const dim3 block(32, kCellTY);
    constexpr int kMaxPlanes = 65535;   // gridDim.z limit: taller grids go in chunks of planes
    const int nz = g->desc.nz, nchunk = (nz + kMaxPlanes - 1) / kMaxPlanes;
    StepArgs<real> a = make_args<real>(g, parity);
    const bool wall = needs_cell_passes(g);   // z walls or a wall sheet
    for (int c = 0; c < nchunk; ++c) {
        a.kbase = c * kMaxPlanes;
        const dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + kCellTY - 1) / kCellTY,
                        nz - a.kbase < kMaxPlanes ? nz - a.kbase : kMaxPlanes);
        if (wall) yee_h_cell_wt<real, kCellTY><<<grid, block, 0, s>>>(a, times, index);
        else yee_h_cell_t<real, kCellTY><<<grid, block, 0, s>>>(a, times, index);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int c = nchunk - 1; c >= 0; --c) {
        a.kbase = c * kMaxPlanes;
        const dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + kCellTY - 1) / kCellTY,
                        nz - a.kbase < kMaxPlanes ? nz - a.kbase : kMaxPlanes);
        if (wall) yee_e_cell_wt<real, kCellTY><<<grid, block, 0, s>>>(a, times, index);
        else yee_e_cell_t<real, kCellTY><<<grid, block, 0, s>>>(a, times, index);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t cell_launch_grid_any(fdtd_batch* b, int q, int parity, int step, cudaStream_t s)
{
    return b->precision == FDTD_F64 ? cell_launch_grid<double>(b, q, parity, step, s)
                                    : cell_launch_grid<float>(b, q, parity, step, s);
}

// One step of every grid on one stream (steps outside a graph replay).
cudaError_t cell_launch_any(fdtd_batch* b, int parity, int step, cudaStream_t s)
{
    for (int q = 0; q < int(b->grids.size()); ++q) {
        cudaError_t e = cell_launch_grid_any(b, q, parity, step, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---- persistent cell engine
template <typename real>
fdtd_status pcell_fill(fdtd_batch* b)
{
    const int n = int(b->grids.size());
    const int ngroups = (n + kPCellGroup - 1) / kPCellGroup;
    char* tab = static_cast<char*>(b->table);
    fdtd_status st = cuda_check(cudaMemset(tab + b->bar_off, 0, kBarBytes), "batch barrier");
    if (st != FDTD_OK) return st;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, yee_batch_cell<real>, 32 * kCellTY, 0);
    if (e != cudaSuccess || per_sm < 1) return fail(FDTD_ECUDA, "persistent cell kernel does not fit on an SM");
    const int sms = b->grids[0]->sm_count > 0 ? b->grids[0]->sm_count : 152;
    b->pc_params.assign(sizeof(PCellParams<real>) * ngroups, 0);
    b->pc_blocks.assign(ngroups, 1);
    for (int gi = 0; gi < ngroups; ++gi) {
        PCellParams<real>& P = reinterpret_cast<PCellParams<real>*>(b->pc_params.data())[gi];
        std::memset(&P, 0, sizeof(P));
        P.q0 = gi * kPCellGroup;
        P.ngrids = n - P.q0 < kPCellGroup ? n - P.q0 : kPCellGroup;
        P.nall = n;
        int blocks = 0;
        for (int q = 0; q < P.ngrids; ++q) {
            const fdtd_grid* g = b->grids[P.q0 + q];
            for (int cur = 0; cur < 2; ++cur) P.args[q][cur] = make_args<real>(g, cur);
            P.ntx[q] = (g->desc.nx + 31) / 32;
            P.nty[q] = (g->desc.ny + kCellTY - 1) / kCellTY;
            P.nz[q] = g->desc.nz;
            P.block0[q] = blocks;
            P.wall[q] = needs_cell_passes(g) ? 1 : 0;
            blocks += P.ntx[q] * P.nty[q] * g->desc.nz;
        }
        P.block0[P.ngrids] = blocks;
        P.nblocks = blocks;
        P.hdr = reinterpret_cast<BatchHeader*>(tab);
        P.times = reinterpret_cast<const StepTime<real>*>(tab + b->times_off);
        P.bar = reinterpret_cast<unsigned*>(tab + b->bar_off);
        // resident CTAs, no more than the barrier words have group counters for
        const int max_ctas = int((kBarBytes / 4 - 4 * kBarLine) / kBarLine) * kBarGroup;
        int ctas = per_sm * sms < blocks ? per_sm * sms : blocks;
        b->pc_blocks[gi] = ctas < max_ctas ? ctas : max_ctas;
    }
    return FDTD_OK;
}

// `count` steps of every grid (time factors already in the table): one
// cooperative launch per group of grids, in order on stream s.
template <typename real>
cudaError_t pcell_launch(fdtd_batch* b, int parity, int count, cudaStream_t s)
{
    for (size_t gi = 0; gi < b->pc_blocks.size(); ++gi) {
        PCellParams<real>& P = reinterpret_cast<PCellParams<real>*>(b->pc_params.data())[gi];
        P.nsteps = count;
        P.parity0 = parity;
        void* args[] = {&P};
        cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(yee_batch_cell<real>),
                                                    dim3(b->pc_blocks[gi]), dim3(32, kCellTY), args, 0, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Time factors of the next `count` steps of every grid into the device table.
template <typename real>
fdtd_status cell_upload_times(fdtd_batch* b, int count)
{
    const int n = int(b->grids.size());
    b->host_times.resize(size_t(count) * n * sizeof(StepTime<real>));
    StepTime<real>* h = reinterpret_cast<StepTime<real>*>(b->host_times.data());
    for (int s = 0; s < count; ++s)
        for (int q = 0; q < n; ++q) {
            const fdtd_grid* g = b->grids[q];
            h[size_t(s) * n + q] = step_time<real>(g->srct, g->has_wall ? &g->wallt : nullptr, g->dt, g->step + s);
        }
    return cuda_check(cudaMemcpyAsync(static_cast<char*>(b->table) + b->times_off, h, b->host_times.size(),
                                      cudaMemcpyHostToDevice, b->stream),
                      "batch time table");
}

// Block shape of the batch: 32 x TR tiles, R rows per thread, S stages
// (FP32: 32 x 8, FP64: 32 x 4, one row per thread, five stages).
template <typename real, int TR, int R, int S>
cudaError_t batch_launch(fdtd_batch* b, int parity, int offset, cudaStream_t s)
{
    using T = TmaTile<real, TR>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(yee_batch_tma<real, TR, R, S>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(T::smem_bytes(S, kBatchLz)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    char* tab = static_cast<char*>(b->table);
    yee_batch_tma<real, TR, R, S><<<b->nblocks, dim3(32, TR / R), T::smem_bytes(S, kBatchLz), s>>>(
        reinterpret_cast<BatchHeader*>(tab), reinterpret_cast<const BatchGrid<real>*>(tab + 256), parity, offset);
    return cudaGetLastError();
}

cudaError_t batch_launch_any(fdtd_batch* b, int parity, int offset, cudaStream_t s)
{
    if (b->precision == FDTD_F64) return batch_launch<double, 4, 1, 5>(b, parity, offset, s);
    return batch_launch<float, 8, 1, 5>(b, parity, offset, s);
}

template <typename real, int TR, int R, int S>
fdtd_status batch_fill(fdtd_batch* b)
{
    using T = TmaTile<real, TR>;
    const int n = int(b->grids.size());
    std::vector<BatchGrid<real>> host(n);
    int items = 0;
    for (int q = 0; q < n; ++q) {
        fdtd_grid* g = b->grids[q];
        BatchGrid<real>& G = host[q];
        std::memset(&G, 0, sizeof(G));
        for (int cur = 0; cur < 2; ++cur) {
            TmaMaps* m = nullptr;
            if (!tma_maps<real, TR>(g, cur, &m)) return fail(FDTD_ECUDA, "tensor map encoding failed");
            G.maps[cur] = *m;
            G.args[cur] = make_args<real>(g, cur);
        }
        G.step0 = g->step;
        G.lz = g->desc.nz < kBatchLz ? g->desc.nz : kBatchLz;
        G.nseg = (g->desc.nz + G.lz - 1) / G.lz;
        G.ntx = (g->desc.nx + 31) / 32;
        G.nty = (g->desc.ny + TR - 1) / TR;
        G.item0 = items;
        items += G.ntx * G.nty * G.nseg;
    }
    b->nitems = items;
    BatchHeader h;
    std::memset(&h, 0, sizeof(h));
    h.ngrids = n;
    h.nitems = items;
    char* tab = static_cast<char*>(b->table);
    fdtd_status st = cuda_check(cudaMemcpy(tab, &h, sizeof(h), cudaMemcpyHostToDevice), "batch table");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpy(tab + 256, host.data(), sizeof(BatchGrid<real>) * n, cudaMemcpyHostToDevice),
                        "batch table");
    if (st != FDTD_OK) return st;
    cudaError_t e = cudaFuncSetAttribute(yee_batch_tma<real, TR, R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(T::smem_bytes(S, kBatchLz)));
    if (e != cudaSuccess) return cuda_check(e, "batch kernel attribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, yee_batch_tma<real, TR, R, S>, 32 * (TR / R),
                                                      T::smem_bytes(S, kBatchLz));
    if (e != cudaSuccess || per_sm < 1) return fail(FDTD_ECUDA, "batch kernel does not fit on an SM");
    const int sms = b->grids[0]->sm_count > 0 ? b->grids[0]->sm_count : 152;
    b->nblocks = per_sm * sms < items ? per_sm * sms : items;
    b->ty = TR;
    b->S = S;
    return FDTD_OK;
}

// The 64 steps of every grid, one branch per grid (streams shared
// round-robin), forked from and joined back into the capture stream.
cudaError_t cell_capture(fdtd_batch* b, int parity)
{
    cudaEvent_t fork, join[kCellBranches];
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    int made = 0;
    for (; made < b->nbranch && e == cudaSuccess; ++made) e = cudaEventCreateWithFlags(&join[made], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(fork, b->capture);
    for (int r = 0; r < b->nbranch && e == cudaSuccess; ++r) {
        e = cudaStreamWaitEvent(b->branch[r], fork, 0);
        for (int q = r; q < int(b->grids.size()) && e == cudaSuccess; q += b->nbranch)
            for (int s = 0; s < kBatchGraphSteps && e == cudaSuccess; ++s)
                e = cell_launch_grid_any(b, q, parity ^ (s & 1), s, b->branch[r]);
        if (e == cudaSuccess) e = cudaEventRecord(join[r], b->branch[r]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->capture, join[r], 0);
    }
    cudaEventDestroy(fork);
    for (int r = 0; r < made; ++r) cudaEventDestroy(join[r]);
    return e;
}

fdtd_status build_graph(fdtd_batch* b, int parity)
{
    cudaGraph_t graph;
    fdtd_status st = cuda_check(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "capture");
    if (st != FDTD_OK) return st;
    cudaError_t e = cudaSuccess;
    if (b->engine == FDTD_BATCH_CELL)
        e = cell_capture(b, parity);
    else
        for (int s = 0; s < kBatchGraphSteps && e == cudaSuccess; ++s)
            e = batch_launch_any(b, parity ^ (s & 1), s, b->capture);
    if (e == cudaSuccess && b->engine == FDTD_BATCH_PERSISTENT) {
        batch_advance<<<1, 1, 0, b->capture>>>(reinterpret_cast<BatchHeader*>(b->table), kBatchGraphSteps);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
    if (e != cudaSuccess) return cuda_check(e, "capture batch launches");
    if (e2 != cudaSuccess) return cuda_check(e2, "end capture");
    e = cudaGraphInstantiate(&b->exec[b->engine][parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_check(e, "graph instantiate");
    b->built[b->engine][parity] = true;
    return FDTD_OK;
}

}  // namespace

extern "C" {

size_t fdtd_batch_required_bytes(int n_grids, int precision)
{
    if (n_grids < 1 || (precision != FDTD_F32 && precision != FDTD_F64)) return 0;
    return times_offset(n_grids, precision) + size_t(kBatchGraphSteps) * n_grids * time_entry_bytes(precision);
}

fdtd_status fdtd_batch_create(fdtd_grid* const* grids, int n, void* dev_table, size_t table_bytes, void* stream,
                              fdtd_batch** out)
{
    if (!out) return fail(FDTD_EINVAL, "null output pointer");
    *out = nullptr;
    if (!grids || n < 1 || !dev_table) return fail(FDTD_EINVAL, "invalid batch arguments");
    if (reinterpret_cast<uintptr_t>(dev_table) % 256 != 0) return fail(FDTD_EINVAL, "table not 256-byte aligned");
    const int prec = grids[0]->desc.precision;
    for (int q = 0; q < n; ++q) {
        if (!grids[q]) return fail(FDTD_EINVAL, "null grid %d", q);
        if (grids[q]->desc.precision != prec) return fail(FDTD_EINVAL, "mixed precisions in one batch");
        if (grids[q]->cur != grids[0]->cur) return fail(FDTD_ESTATE, "grids must start from the same copy parity");
        const fdtd_status dev_st = check_device(grids[q], "fdtd_batch_create");
        if (dev_st != FDTD_OK) return dev_st;
    }
    if (table_bytes < fdtd_batch_required_bytes(n, prec))
        return fail(FDTD_ENOMEM, "batch table of %zu bytes, %zu needed", table_bytes, fdtd_batch_required_bytes(n, prec));
    fdtd_batch* b = new (std::nothrow) fdtd_batch();
    if (!b) return fail(FDTD_ENOMEM, "host allocation failed");
    b->grids.assign(grids, grids + n);
    b->precision = prec;
    b->table = dev_table;
    b->table_bytes = table_bytes;
    b->stream = static_cast<cudaStream_t>(stream);
    b->cur = grids[0]->cur;
    b->step = 0;
    b->engine = FDTD_BATCH_CELL;
    b->times_off = times_offset(n, prec);
    b->bar_off = bar_offset(n, prec);
    for (int e = 0; e < 2; ++e) b->built[e][0] = b->built[e][1] = false;
    fdtd_status st = cuda_check(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream");
    if (st != FDTD_OK) { delete b; return st; }
    st = cuda_check(cudaStreamSynchronize(b->stream), "batch create");
    if (st == FDTD_OK) st = prec == FDTD_F64 ? batch_fill<double, 4, 1, 5>(b) : batch_fill<float, 8, 1, 5>(b);
    if (st != FDTD_OK) { cudaStreamDestroy(b->capture); delete b; return st; }
    cell_fill(b);
    if (st == FDTD_OK) st = prec == FDTD_F64 ? pcell_fill<double>(b) : pcell_fill<float>(b);
    if (st != FDTD_OK) { cudaStreamDestroy(b->capture); delete b; return st; }
    b->nbranch = n < kCellBranches ? n : kCellBranches;
    for (int r = 0; r < b->nbranch && st == FDTD_OK; ++r) {
        st = cuda_check(cudaStreamCreateWithFlags(&b->branch[r], cudaStreamNonBlocking), "branch stream");
        if (st != FDTD_OK) {
            for (int q = 0; q < r; ++q) cudaStreamDestroy(b->branch[q]);
            cudaStreamDestroy(b->capture);
            delete b;
            return st;
        }
    }
    for (fdtd_grid* g : b->grids) ++g->batch_refs;
    *out = b;
    return FDTD_OK;
}

fdtd_status fdtd_batch_set_engine(fdtd_batch* b, int engine)
{
    if (!b) return fail(FDTD_EINVAL, "null batch");
    if (engine != FDTD_BATCH_PERSISTENT && engine != FDTD_BATCH_CELL && engine != FDTD_BATCH_PERSISTENT_CELL)
        return fail(FDTD_EINVAL, "engine %d is not FDTD_BATCH_PERSISTENT, _CELL or _PERSISTENT_CELL", engine);
    if (engine == FDTD_BATCH_PERSISTENT)
        for (fdtd_grid* g : b->grids)
            if (needs_cell_passes(g))
                return fail(FDTD_EINVAL, "the persistent engine takes z-periodic grids without a wall source");
    if (engine == FDTD_BATCH_PERSISTENT && b->engine != engine) {
        // the persistent kernel takes the source phase of grid g at step
        // step0_g + counter: bring the device counter to the batch's step
        const long long counter = b->step;
        fdtd_status st = cuda_check(cudaMemcpyAsync(static_cast<char*>(b->table) + offsetof(BatchHeader, counter),
                                                    &counter, sizeof(counter), cudaMemcpyHostToDevice, b->stream),
                                    "batch counter");
        if (st != FDTD_OK) return st;
        st = cuda_check(cudaStreamSynchronize(b->stream), "batch counter");
        if (st != FDTD_OK) return st;
    }
    b->engine = engine;
    return FDTD_OK;
}

int fdtd_batch_get_engine(const fdtd_batch* b) { return b ? b->engine : -1; }

fdtd_status fdtd_batch_debug_inject_fault(fdtd_batch* b, int kind)
{
    if (!b) return fail(FDTD_EINVAL, "null batch");
    if (kind != 0 && kind != 1) return fail(FDTD_EINVAL, "fault kind %d not in {0, 1}", kind);
    fdtd_status st = cuda_check(cudaMemcpyAsync(static_cast<char*>(b->table) + offsetof(BatchHeader, fault), &kind,
                                                sizeof(int), cudaMemcpyHostToDevice, b->stream), "fault hook");
    if (st == FDTD_OK) st = cuda_check(cudaStreamSynchronize(b->stream), "fault hook");
    if (st == FDTD_OK) b->fault = kind;
    return st;
}

static fdtd_status batch_step_ranges(fdtd_batch* b, int nsteps);

fdtd_status fdtd_batch_step(fdtd_batch* b, int nsteps)
{
    nvtxRangePushA("fdtd_batch_step");
    fdtd_status st = batch_step_ranges(b, nsteps);
    nvtxRangePop();
    return st;
}

static fdtd_status batch_step_ranges(fdtd_batch* b, int nsteps)
{
    if (!b || nsteps < 0) return fail(FDTD_EINVAL, "invalid argument");
    const fdtd_status dev_st = check_device(b->grids[0], "fdtd_batch_step");
    if (dev_st != FDTD_OK) return dev_st;
    for (fdtd_grid* g : b->grids)
        if (g->cur != b->cur) return fail(FDTD_ESTATE, "a batched grid was stepped outside the batch");
    const bool cell = b->engine == FDTD_BATCH_CELL;
    int done = 0;
    if (b->engine == FDTD_BATCH_PERSISTENT_CELL) {
        while (done < nsteps) {
            const int count = nsteps - done < kBatchGraphSteps ? nsteps - done : kBatchGraphSteps;
            fdtd_status st = b->precision == FDTD_F64 ? cell_upload_times<double>(b, count)
                                                      : cell_upload_times<float>(b, count);
            if (st != FDTD_OK) return st;
            cudaError_t e = b->precision == FDTD_F64 ? pcell_launch<double>(b, b->cur, count, b->stream)
                                                     : pcell_launch<float>(b, b->cur, count, b->stream);
            if (e != cudaSuccess) return cuda_check(e, "persistent cell launch");
            if (b->fault) {   // the hook applies to one launch
                static const int zero = 0;
                e = cudaMemcpyAsync(static_cast<char*>(b->table) + offsetof(BatchHeader, fault), &zero, sizeof(int),
                                    cudaMemcpyHostToDevice, b->stream);
                if (e != cudaSuccess) return cuda_check(e, "clear fault hook");
                b->fault = 0;
            }
            b->cur ^= (count & 1);
            done += count;
            b->step += count;
            for (fdtd_grid* g : b->grids) {
                g->step += count;
                g->cur = b->cur;
            }
        }
        return FDTD_OK;
    }
    while (done < nsteps) {
        const int count = nsteps - done < kBatchGraphSteps ? nsteps - done : kBatchGraphSteps;
        if (cell) {
            fdtd_status st = b->precision == FDTD_F64 ? cell_upload_times<double>(b, count)
                                                      : cell_upload_times<float>(b, count);
            if (st != FDTD_OK) return st;
        }
        if (count == kBatchGraphSteps) {
            if (!b->built[b->engine][b->cur]) {
                fdtd_status st = build_graph(b, b->cur);
                if (st != FDTD_OK) return st;
            }
            fdtd_status st = cuda_check(cudaGraphLaunch(b->exec[b->engine][b->cur], b->stream), "graph launch");
            if (st != FDTD_OK) return st;
        } else {
            for (int s = 0; s < count; ++s) {
                cudaError_t e = cell ? cell_launch_any(b, b->cur ^ (s & 1), s, b->stream)
                                     : batch_launch_any(b, b->cur ^ (s & 1), s, b->stream);
                if (e != cudaSuccess) return cuda_check(e, "batch launch");
            }
            if (!cell) {
                batch_advance<<<1, 1, 0, b->stream>>>(reinterpret_cast<BatchHeader*>(b->table), count);
                fdtd_status st = cuda_check(cudaGetLastError(), "batch advance");
                if (st != FDTD_OK) return st;
            }
            b->cur ^= (count & 1);
        }
        done += count;
        b->step += count;
        for (fdtd_grid* g : b->grids) {
            g->step += count;
            g->cur = b->cur;
        }
    }
    return FDTD_OK;
}

fdtd_status fdtd_batch_sync(fdtd_batch* b)
{
    if (!b) return fail(FDTD_EINVAL, "null batch");
    const fdtd_status dev_st = check_device(b->grids[0], "fdtd_batch_sync");
    if (dev_st != FDTD_OK) return dev_st;
    fdtd_status st = cuda_check(cudaStreamSynchronize(b->stream), "batch synchronize");
    if (st != FDTD_OK) return st;
    BatchHeader h;
    st = cuda_check(cudaMemcpy(&h, b->table, sizeof(h), cudaMemcpyDeviceToHost), "read batch header");
    if (st != FDTD_OK) return st;
    if (h.err != 0) {
        int zero = 0;
        cudaMemcpy(static_cast<char*>(b->table) + offsetof(BatchHeader, err), &zero, sizeof(int),
                   cudaMemcpyHostToDevice);
        // an expired grid barrier may have left its arrival count part-way
        cudaMemset(static_cast<char*>(b->table) + b->bar_off, 0, kBarBytes);
        return fail(FDTD_ETIMEOUT, "a bounded device-side wait expired in the batched step");
    }
    return FDTD_OK;
}

int fdtd_batch_work_items(const fdtd_batch* b)
{
    if (!b) return -1;
    return b->engine == FDTD_BATCH_PERSISTENT ? b->nitems : b->cell_blocks;
}

void fdtd_batch_destroy(fdtd_batch* b)
{
    if (!b) return;
    for (fdtd_grid* g : b->grids) --g->batch_refs;
    for (int e = 0; e < 2; ++e)
        for (int p = 0; p < 2; ++p)
            if (b->built[e][p]) cudaGraphExecDestroy(b->exec[e][p]);
    for (int r = 0; r < b->nbranch; ++r) cudaStreamDestroy(b->branch[r]);
    cudaStreamDestroy(b->capture);
    delete b;
}

}  // extern "C"
