// batch.cu -- many independent Bessel-antenna grids (different orders, cone
// angles, ring radii and transverse sizes) advanced together.
//
// Each grid runs the unchanged method of its own descriptor (Section 4,
// Eq. 12-13).  Two engines:
//   * graph (FDTD_BATCH_CELL, the default): a CUDA graph holds K = 64
//     consecutive steps of every grid, one branch per grid (up to
//     kCellBranches concurrent streams, shared round-robin), so that the
//     launches of small grids run side by side instead of each leaving the
//     GPU idle in its tail.  Each grid steps in its own mode: the
//     cell-parallel H and E passes of tile variant 5 on 32 x 4, 8 or 16
//     blocks, or (FP32 z-periodic grids without a wall sheet) the two-step
//     kernel of tile variant 7 on a share of the SMs proportional to its
//     cells.  The per-step source time factors of every grid are evaluated on
//     the host in FP64, as for a single grid, and copied into a device table
//     ahead of each replay; the kernels read their steps' entries.
//   * persistent cell passes (FDTD_BATCH_PERSISTENT_CELL): one cooperative
//     kernel launch runs up to K steps of every grid.  The 32 x 4 cell
//     blocks of all grids form one list; the CTAs (one per resident slot)
//     take runs of kPCellChunk consecutive blocks, in order, from a per-pass
//     counter (the E pass from the end of the list), then single blocks near
//     the end of the pass, so that the blocks in flight stay a narrow front
//     whose neighbours are in L2, as under the hardware block scheduler, and
//     a pass ends within about one block of its average.  H pass of every
//     grid, grid barrier, E pass, barrier, and so on.  The cell arithmetic is
//     that of tile variant 5, bit for bit; the barriers are bounded waits.
// fdtd_batch_autotune picks each grid's cell-pass block height alone, then
// times the whole batch with the grids above each size threshold on the
// two-step kernel (on proportional shares of the SMs or on all of them) and
// on the persistent cell engine, keeps the fastest, and restores every
// grid's state.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "grid_impl.h"
#include "yee_cell.cuh"

namespace fdtd {

struct BatchHeader {
    int ngrids;
    int err;             // device error word
    int fault;           // test hook: 1 = CTA 0 of the next persistent cell launch never arrives
};

constexpr int kBatchGraphSteps = 64;   // even, so a replay leaves the read copy unchanged

// ---- graph engine
constexpr int kCellTY = 4;          // 32 x 4 x 1 cell blocks (tile variant 5) of the persistent cell engine
constexpr int kCellBranches = 16;   // concurrent graph branches (grids share them round-robin)
// Per-grid modes of the graph engine.
enum { kModeCell4 = 0, kModeCell8 = 1, kModeCell16 = 2, kModeTwoStep = 3 };

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
    int engine;                      // FDTD_BATCH_CELL or FDTD_BATCH_PERSISTENT_CELL
    void* table;
    size_t table_bytes;
    size_t times_off;                // byte offset of the time table in `table`
    size_t bar_off;                  // byte offset of the persistent engine's barrier words
    cudaStream_t stream;
    cudaStream_t capture;
    int cell_blocks;                 // 32 x 4 cell blocks per step and pass
    std::vector<unsigned char> pc_params;   // persistent cell engine: PCellParams of each group
    std::vector<int> pc_blocks;             // resident CTAs of each group's launch
    int fault;                       // fdtd_batch_debug_inject_fault pending
    cudaStream_t branch[kCellBranches];
    int nbranch;
    std::vector<unsigned char> host_times;
    std::vector<int> mode;           // graph engine: each grid's mode (kModeCell4 ... kModeTwoStep)
    std::vector<int> ctas;           // two-step mode: CTAs of the grid's launches
    bool shared_sms;                 // two-step launches on proportional shares of the SMs (else all)
    int cur;
    int64_t step;
    cudaGraphExec_t exec[2];         // graph engine, by read copy at the replay's start
    bool built[2];
};

namespace {

size_t time_entry_bytes(int precision)
{
    return precision == FDTD_F64 ? sizeof(StepTime<double>) : sizeof(StepTime<float>);
}

// Table layout: header (256 B) | barrier words (kBarBytes) | time factors.
size_t bar_offset() { return 256; }

size_t times_offset() { return bar_offset() + kBarBytes; }

void cell_fill(fdtd_batch* b)
{
    b->cell_blocks = 0;
    for (const fdtd_grid* g : b->grids)
        b->cell_blocks += ((g->desc.nx + 31) / 32) * ((g->desc.ny + kCellTY - 1) / kCellTY) * g->desc.nz;
}

// Step `step` of the replay for grid q on stream s with the cell passes on
// 32 x TY blocks (time factor times[step * n + q]).
template <typename real, int TY>
cudaError_t cell_launch_grid(fdtd_batch* b, int q, int parity, int step, cudaStream_t s)
{
    const fdtd_grid* g = b->grids[q];
    const StepTime<real>* times =
        reinterpret_cast<const StepTime<real>*>(static_cast<char*>(b->table) + b->times_off);
    const int index = step * int(b->grids.size()) + q;
    const dim3 block(32, TY);
    constexpr int kMaxPlanes = 65535;   // gridDim.z limit: taller grids go in chunks of planes
    const int nz = g->desc.nz, nchunk = (nz + kMaxPlanes - 1) / kMaxPlanes;
    StepArgs<real> a = make_args<real>(g, parity);
    const bool wall = needs_cell_passes(g);   // z walls or a wall sheet
    for (int c = 0; c < nchunk; ++c) {
        a.kbase = c * kMaxPlanes;
        const dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TY - 1) / TY,
                        nz - a.kbase < kMaxPlanes ? nz - a.kbase : kMaxPlanes);
        if (wall) yee_h_cell_wt<real, TY><<<grid, block, 0, s>>>(a, times, index);
        else yee_h_cell_t<real, TY><<<grid, block, 0, s>>>(a, times, index);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int c = nchunk - 1; c >= 0; --c) {
        a.kbase = c * kMaxPlanes;
        const dim3 grid((g->desc.nx + 31) / 32, (g->desc.ny + TY - 1) / TY,
                        nz - a.kbase < kMaxPlanes ? nz - a.kbase : kMaxPlanes);
        if (wall) yee_e_cell_wt<real, TY><<<grid, block, 0, s>>>(a, times, index);
        else yee_e_cell_t<real, TY><<<grid, block, 0, s>>>(a, times, index);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One step of grid q with the cell passes of its mode (the two-step mode
// takes single steps on 32 x 4 blocks).
cudaError_t cell_launch_grid_any(fdtd_batch* b, int q, int parity, int step, cudaStream_t s)
{
    const int m = b->mode[size_t(q)];
    if (b->precision == FDTD_F64) {
        if (m == kModeCell8) return cell_launch_grid<double, 8>(b, q, parity, step, s);
        if (m == kModeCell16) return cell_launch_grid<double, 16>(b, q, parity, step, s);
        return cell_launch_grid<double, 4>(b, q, parity, step, s);
    }
    if (m == kModeCell8) return cell_launch_grid<float, 8>(b, q, parity, step, s);
    if (m == kModeCell16) return cell_launch_grid<float, 16>(b, q, parity, step, s);
    return cell_launch_grid<float, 4>(b, q, parity, step, s);
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

// The K steps of grid q in the graph: K / 2 two-step launches (copies and
// E-side psi flip once per launch; K / 2 is even, so a replay leaves both as
// they were) or K single steps.
cudaError_t graph_grid(fdtd_batch* b, int q, int parity, cudaStream_t s)
{
    if (b->mode[size_t(q)] == kModeTwoStep) {
        const StepTime<float>* times =
            reinterpret_cast<const StepTime<float>*>(static_cast<char*>(b->table) + b->times_off);
        const int n = int(b->grids.size());
        fdtd_grid* g = b->grids[size_t(q)];
        const int pe0 = g->pe;
        cudaError_t e = cudaSuccess;
        for (int l = 0; l < kBatchGraphSteps / 2 && e == cudaSuccess; ++l) {
            g->pe = pe0 ^ (l & 1);   // make_args picks the E-side psi copy of this launch
            e = launch_tb2_table(g, parity ^ (l & 1), times, 2 * l * n + q, (2 * l + 1) * n + q,
                                 b->ctas[size_t(q)], s);
        }
        g->pe = pe0;
        return e;
    }
    for (int st = 0; st < kBatchGraphSteps; ++st) {
        cudaError_t e = cell_launch_grid_any(b, q, parity ^ (st & 1), st, s);
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

// The K steps of every grid, one branch per grid (streams shared
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
        for (int q = r; q < int(b->grids.size()) && e == cudaSuccess; q += b->nbranch) e = graph_grid(b, q, parity, b->branch[r]);
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
    cudaError_t e = cell_capture(b, parity);
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
    if (e != cudaSuccess) return cuda_check(e, "capture batch launches");
    if (e2 != cudaSuccess) return cuda_check(e2, "end capture");
    e = cudaGraphInstantiate(&b->exec[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_check(e, "graph instantiate");
    b->built[parity] = true;
    return FDTD_OK;
}

void drop_graphs(fdtd_batch* b)
{
    for (int p = 0; p < 2; ++p)
        if (b->built[p]) {
            cudaGraphExecDestroy(b->exec[p]);
            b->built[p] = false;
        }
}

// CTAs of grid q's two-step launches: with `shared`, a share of the
// resident slots proportional to its cells, so that the grids' launches run
// side by side; otherwise every slot, each launch filling the SMs its
// predecessors free as they finish.
void two_step_ctas(fdtd_batch* b, bool shared)
{
    double total = 0.0;
    for (const fdtd_grid* g : b->grids) total += double(g->desc.nx) * g->desc.ny * g->desc.nz;
    const int sms = b->grids[0]->sm_count > 0 ? b->grids[0]->sm_count : 152;
    b->ctas.assign(b->grids.size(), sms);
    b->shared_sms = shared;
    if (!shared) return;
    for (size_t q = 0; q < b->grids.size(); ++q) {
        const fdtd_grid* g = b->grids[q];
        const double share = double(g->desc.nx) * g->desc.ny * g->desc.nz / total;
        b->ctas[q] = std::max(8, std::min(sms, int(share * sms + 0.5)));
    }
}

bool two_step_eligible(const fdtd_batch* b, int q)
{
    return b->precision == FDTD_F32 && !needs_cell_passes(b->grids[size_t(q)]);
}

}  // namespace

extern "C" {

size_t fdtd_batch_required_bytes(int n_grids, int precision)
{
    if (n_grids < 1 || (precision != FDTD_F32 && precision != FDTD_F64)) return 0;
    return times_offset() + size_t(kBatchGraphSteps) * n_grids * time_entry_bytes(precision);
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
    b->times_off = times_offset();
    b->bar_off = bar_offset();
    b->fault = 0;
    b->mode.assign(size_t(n), kModeCell4);
    two_step_ctas(b, true);
    b->built[0] = b->built[1] = false;
    fdtd_status st = cuda_check(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream");
    if (st != FDTD_OK) { delete b; return st; }
    BatchHeader h;
    std::memset(&h, 0, sizeof(h));
    h.ngrids = n;
    st = cuda_check(cudaStreamSynchronize(b->stream), "batch create");
    if (st == FDTD_OK) st = cuda_check(cudaMemcpy(b->table, &h, sizeof(h), cudaMemcpyHostToDevice), "batch table");
    if (st != FDTD_OK) { cudaStreamDestroy(b->capture); delete b; return st; }
    cell_fill(b);
    st = prec == FDTD_F64 ? pcell_fill<double>(b) : pcell_fill<float>(b);
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
    if (engine == FDTD_BATCH_PERSISTENT)
        return fail(FDTD_EINVAL, "the persistent TMA batch engine is no longer built (it ran slower than the "
                                 "grids stepped one by one); use FDTD_BATCH_CELL or FDTD_BATCH_PERSISTENT_CELL");
    if (engine != FDTD_BATCH_CELL && engine != FDTD_BATCH_PERSISTENT_CELL)
        return fail(FDTD_EINVAL, "engine %d is not FDTD_BATCH_CELL or FDTD_BATCH_PERSISTENT_CELL", engine);
    b->engine = engine;
    return FDTD_OK;
}

int fdtd_batch_get_engine(const fdtd_batch* b) { return b ? b->engine : -1; }

fdtd_status fdtd_batch_set_grid_mode(fdtd_batch* b, int q, int mode)
{
    if (!b || q < 0 || q >= int(b->grids.size())) return fail(FDTD_EINVAL, "invalid batch or grid index");
    if (mode < FDTD_BATCH_MODE_CELL4 || mode > FDTD_BATCH_MODE_TWO_STEP)
        return fail(FDTD_EINVAL, "mode %d is not a batch grid mode", mode);
    if (mode == FDTD_BATCH_MODE_TWO_STEP && !two_step_eligible(b, q))
        return fail(FDTD_EINVAL, "the two-step mode takes FP32 z-periodic grids without a wall source");
    if (b->mode[size_t(q)] != mode) {
        b->mode[size_t(q)] = mode;
        drop_graphs(b);
    }
    return FDTD_OK;
}

int fdtd_batch_get_grid_mode(const fdtd_batch* b, int q)
{
    if (!b || q < 0 || q >= int(b->grids.size())) return -1;
    return b->mode[size_t(q)];
}

int fdtd_batch_get_grid_ctas(const fdtd_batch* b, int q)
{
    if (!b || q < 0 || q >= int(b->grids.size())) return -1;
    return b->ctas[size_t(q)];
}

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
    int done = 0;
    while (done < nsteps) {
        const int count = nsteps - done < kBatchGraphSteps ? nsteps - done : kBatchGraphSteps;
        fdtd_status st = b->precision == FDTD_F64 ? cell_upload_times<double>(b, count)
                                                  : cell_upload_times<float>(b, count);
        if (st != FDTD_OK) return st;
        if (b->engine == FDTD_BATCH_PERSISTENT_CELL) {
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
        } else if (count == kBatchGraphSteps) {
            if (!b->built[b->cur]) {
                st = build_graph(b, b->cur);
                if (st != FDTD_OK) return st;
            }
            st = cuda_check(cudaGraphLaunch(b->exec[b->cur], b->stream), "graph launch");
            if (st != FDTD_OK) return st;
        } else {
            for (int s = 0; s < count; ++s) {
                cudaError_t e = cell_launch_any(b, b->cur ^ (s & 1), s, b->stream);
                if (e != cudaSuccess) return cuda_check(e, "batch launch");
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

int fdtd_batch_work_items(const fdtd_batch* b) { return b ? b->cell_blocks : -1; }

size_t fdtd_batch_autotune_bytes(const fdtd_batch* b)
{
    if (!b) return 0;
    size_t total = 0;
    for (const fdtd_grid* g : b->grids) total += (fdtd_state_bytes(g) + 255) / 256 * 256;
    return total;
}

// Saves every grid (scratch: fdtd_batch_autotune_bytes), times each grid's
// modes alone, then the two engines over the whole batch, restores every grid
// and keeps the fastest.
fdtd_status fdtd_batch_autotune(fdtd_batch* b, int steps, void* scratch, size_t scratch_bytes)
{
    if (!b || !scratch || steps < 1) return fail(FDTD_EINVAL, "invalid argument");
    const fdtd_status dev_st = check_device(b->grids[0], "fdtd_batch_autotune");
    if (dev_st != FDTD_OK) return dev_st;
    if (scratch_bytes < fdtd_batch_autotune_bytes(b))
        return fail(FDTD_ENOMEM, "autotune scratch of %zu bytes, %zu needed", scratch_bytes, fdtd_batch_autotune_bytes(b));
    const int n = int(b->grids.size());
    std::vector<size_t> offs(static_cast<size_t>(n), 0);
    size_t o = 0;
    for (int q = 0; q < n; ++q) {
        offs[size_t(q)] = o;
        o += (fdtd_state_bytes(b->grids[size_t(q)]) + 255) / 256 * 256;
    }
    char* S = static_cast<char*>(scratch);
    const int64_t step0 = b->step;
    const int cur0 = b->cur;
    auto save_all = [&]() {
        for (int q = 0; q < n; ++q) {
            fdtd_grid* g = b->grids[size_t(q)];
            const int refs = g->batch_refs;
            g->batch_refs = 0;
            fdtd_status st = fdtd_save_state(g, S + offs[size_t(q)]);
            g->batch_refs = refs;
            if (st != FDTD_OK) return st;
        }
        return FDTD_OK;
    };
    auto load_all = [&]() {
        for (int q = 0; q < n; ++q) {
            fdtd_grid* g = b->grids[size_t(q)];
            fdtd_status st = fdtd_load_state(g, S + offs[size_t(q)]);
            if (st != FDTD_OK) return st;
        }
        b->step = step0;
        b->cur = cur0;
        return FDTD_OK;
    };
    fdtd_status st = save_all();
    if (st != FDTD_OK) return st;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(FDTD_ECUDA, "event create failed");
    const int nrun = steps + (steps & 1);
    auto elapsed = [&]() {
        float ms = 0.0f;
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // 1. each grid alone on the cell passes of each block height, single-grid
    //    launches on the batch stream: its cell mode
    cudaError_t err = cudaSuccess;
    std::vector<int> cell_mode(size_t(n), kModeCell4);
    for (int q = 0; q < n && err == cudaSuccess; ++q) {
        fdtd_grid* g = b->grids[size_t(q)];
        const int refs = g->batch_refs;
        g->batch_refs = 0;
        const cudaStream_t gs = g->stream;
        const TileConfig keep = g->tile;
        g->stream = b->stream;
        float best = 1e30f;
        for (int m = kModeCell4; m <= kModeCell16 && err == cudaSuccess; ++m) {
            TileConfig tc = keep;
            tc.variant = 5;
            tc.ty = m == kModeCell8 ? 8 : (m == kModeCell16 ? 16 : 4);
            g->tile = tc;
            if (fdtd_step(g, 2) != FDTD_OK) err = cudaErrorUnknown;   // warm-up
            cudaEventRecord(e0, b->stream);
            if (err == cudaSuccess && fdtd_step(g, nrun) != FDTD_OK) err = cudaErrorUnknown;
            cudaEventRecord(e1, b->stream);
            const float ms = elapsed();
            if (err == cudaSuccess && ms < best) { best = ms; cell_mode[size_t(q)] = m; }
        }
        g->tile = keep;
        g->stream = gs;
        g->batch_refs = refs;
        if (fdtd_load_state(g, S + offs[size_t(q)]) != FDTD_OK && err == cudaSuccess) err = cudaErrorUnknown;
    }
    // 2. the whole batch, kBatchGraphSteps steps after a warm-up replay, best
    //    of two: the graph with the grids of at least `thr` cells on the
    //    two-step kernel (thr over every eligible grid's size, and none), on
    //    shares of the SMs or on all of them; the persistent cell engine
    std::vector<long long> thresholds = {-1};   // -1: no grid on the two-step kernel
    for (int q = 0; q < n; ++q)
        if (two_step_eligible(b, q)) {
            const fdtd_grid* g = b->grids[size_t(q)];
            const long long c = (long long)g->desc.nx * g->desc.ny * g->desc.nz;
            if (std::find(thresholds.begin(), thresholds.end(), c) == thresholds.end()) thresholds.push_back(c);
        }
    auto apply = [&](long long thr) {
        for (int q = 0; q < n; ++q) {
            const fdtd_grid* g = b->grids[size_t(q)];
            const long long c = (long long)g->desc.nx * g->desc.ny * g->desc.nz;
            b->mode[size_t(q)] = (thr >= 0 && c >= thr && two_step_eligible(b, q)) ? kModeTwoStep : cell_mode[size_t(q)];
        }
        drop_graphs(b);
    };
    auto time_batch = [&](float* out) {
        float best = 1e30f;
        st = fdtd_batch_step(b, kBatchGraphSteps);   // warm-up (builds the graph)
        for (int rep = 0; rep < 2 && st == FDTD_OK; ++rep) {
            cudaEventRecord(e0, b->stream);
            st = fdtd_batch_step(b, kBatchGraphSteps);
            cudaEventRecord(e1, b->stream);
            const float ms = elapsed();
            if (ms < best) best = ms;
        }
        if (st == FDTD_OK) st = fdtd_batch_sync(b);
        if (st == FDTD_OK) st = load_all();
        *out = best;
        return st == FDTD_OK;
    };
    const int keep_engine = b->engine;
    float best_t = 1e30f;
    long long best_thr = -1;
    bool best_shared = true;
    int best_engine = FDTD_BATCH_CELL;
    b->engine = FDTD_BATCH_CELL;
    for (long long thr : thresholds) {
        for (int sh = 0; sh < 2 && err == cudaSuccess; ++sh) {
            if (thr < 0 && sh == 1) break;   // no two-step grid: the shares do not matter
            apply(thr);
            two_step_ctas(b, sh == 0);
            float t = 0.0f;
            if (!time_batch(&t)) { err = cudaErrorUnknown; break; }
            if (t < best_t) { best_t = t; best_thr = thr; best_shared = sh == 0; best_engine = FDTD_BATCH_CELL; }
        }
        if (err != cudaSuccess) break;
    }
    if (err == cudaSuccess) {
        b->engine = FDTD_BATCH_PERSISTENT_CELL;
        float t = 0.0f;
        if (!time_batch(&t)) err = cudaErrorUnknown;
        else if (t < best_t) { best_t = t; best_engine = FDTD_BATCH_PERSISTENT_CELL; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err == cudaSuccess) {
        b->engine = best_engine;
        apply(best_thr);
        two_step_ctas(b, best_shared);
    } else {
        b->engine = keep_engine;
        apply(-1);
    }
    const fdtd_status rst = load_all();
    if (err != cudaSuccess) return st != FDTD_OK ? st : fail(FDTD_ECUDA, "batch autotune failed: %s", fdtd_last_error());
    return rst;
}

void fdtd_batch_destroy(fdtd_batch* b)
{
    if (!b) return;
    for (fdtd_grid* g : b->grids) --g->batch_refs;
    drop_graphs(b);
    for (int r = 0; r < b->nbranch; ++r) cudaStreamDestroy(b->branch[r]);
    cudaStreamDestroy(b->capture);
    delete b;
}

}  // extern "C"
