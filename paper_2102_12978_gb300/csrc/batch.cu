// batch.cu -- many independent Bessel-antenna grids (different orders, cone
// angles, ring radii and transverse sizes) advanced together.
//
// Each grid runs the unchanged method of its own descriptor (Section 4,
// Eq. 12-13).  The batch flattens every grid's (32 x TR tile, z segment)
// blocks into one work list; a persistent kernel with one CTA per resident
// slot (SM count x occupancy) walks the list with a grid stride, marching
// each block with the TMA-staged fused step (tma_march).  The CTA's
// mbarriers are initialised once and their phases carried from block to
// block.  A CUDA graph holds K consecutive step launches plus a one-thread
// kernel that advances the batch's device step counter, so one graph replay
// advances every grid by K steps and the source phase of step n stays
// correct on every replay.
#include <cuda_runtime.h>

#include <cstring>
#include <new>
#include <vector>

#include "../../include/fdtd.h"
#include "grid_impl.h"
#include "tma_host.h"
#include "yee_tma.cuh"

namespace fdtd {

struct BatchHeader {
    int ngrids, nitems;
    long long counter;   // steps taken by the batch since creation
    int err;             // device error word
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

}  // namespace fdtd

using namespace fdtd;

struct fdtd_batch {
    std::vector<fdtd_grid*> grids;
    int precision;
    int ty, S;
    void* table;
    size_t table_bytes;
    cudaStream_t stream;
    cudaStream_t capture;
    int nitems;
    int nblocks;
    int cur;
    int64_t step;
    cudaGraphExec_t exec[2];
    bool built[2];
};

namespace {

size_t grid_entry_bytes(int precision)
{
    return precision == FDTD_F64 ? sizeof(BatchGrid<double>) : sizeof(BatchGrid<float>);
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

fdtd_status build_graph(fdtd_batch* b, int parity)
{
    cudaGraph_t graph;
    fdtd_status st = cuda_check(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "capture");
    if (st != FDTD_OK) return st;
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < kBatchGraphSteps && e == cudaSuccess; ++s)
        e = batch_launch_any(b, parity ^ (s & 1), s, b->capture);
    if (e == cudaSuccess) {
        batch_advance<<<1, 1, 0, b->capture>>>(reinterpret_cast<BatchHeader*>(b->table), kBatchGraphSteps);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
    if (e != cudaSuccess) return cuda_check(e, "capture batch launches");
    if (e2 != cudaSuccess) return cuda_check(e2, "end capture");
    e = cudaGraphInstantiate(&b->exec[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_check(e, "graph instantiate");
    b->built[parity] = true;
    return FDTD_OK;
}

}  // namespace

extern "C" {

size_t fdtd_batch_required_bytes(int n_grids, int precision)
{
    if (n_grids < 1 || (precision != FDTD_F32 && precision != FDTD_F64)) return 0;
    return 256 + grid_entry_bytes(precision) * size_t(n_grids);
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
    b->built[0] = b->built[1] = false;
    fdtd_status st = cuda_check(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream");
    if (st != FDTD_OK) { delete b; return st; }
    st = cuda_check(cudaStreamSynchronize(b->stream), "batch create");
    if (st == FDTD_OK) st = prec == FDTD_F64 ? batch_fill<double, 4, 1, 5>(b) : batch_fill<float, 8, 1, 5>(b);
    if (st != FDTD_OK) { cudaStreamDestroy(b->capture); delete b; return st; }
    *out = b;
    return FDTD_OK;
}

fdtd_status fdtd_batch_step(fdtd_batch* b, int nsteps)
{
    if (!b || nsteps < 0) return fail(FDTD_EINVAL, "invalid argument");
    for (fdtd_grid* g : b->grids)
        if (g->cur != b->cur) return fail(FDTD_ESTATE, "a batched grid was stepped outside the batch");
    const int full = nsteps / kBatchGraphSteps, rem = nsteps % kBatchGraphSteps;
    for (int r = 0; r < full; ++r) {
        if (!b->built[b->cur]) {
            fdtd_status st = build_graph(b, b->cur);
            if (st != FDTD_OK) return st;
        }
        fdtd_status st = cuda_check(cudaGraphLaunch(b->exec[b->cur], b->stream), "graph launch");
        if (st != FDTD_OK) return st;
    }
    for (int s = 0; s < rem; ++s) {
        cudaError_t e = batch_launch_any(b, b->cur ^ (s & 1), s, b->stream);
        if (e != cudaSuccess) return cuda_check(e, "batch launch");
    }
    if (rem > 0) {
        batch_advance<<<1, 1, 0, b->stream>>>(reinterpret_cast<BatchHeader*>(b->table), rem);
        fdtd_status st = cuda_check(cudaGetLastError(), "batch advance");
        if (st != FDTD_OK) return st;
        b->cur ^= (rem & 1);
    }
    b->step += nsteps;
    for (fdtd_grid* g : b->grids) {
        g->step += nsteps;
        g->cur = b->cur;
    }
    return FDTD_OK;
}

fdtd_status fdtd_batch_sync(fdtd_batch* b)
{
    if (!b) return fail(FDTD_EINVAL, "null batch");
    fdtd_status st = cuda_check(cudaStreamSynchronize(b->stream), "batch synchronize");
    if (st != FDTD_OK) return st;
    BatchHeader h;
    st = cuda_check(cudaMemcpy(&h, b->table, sizeof(h), cudaMemcpyDeviceToHost), "read batch header");
    if (st != FDTD_OK) return st;
    if (h.err != 0) {
        int zero = 0;
        cudaMemcpy(static_cast<char*>(b->table) + offsetof(BatchHeader, err), &zero, sizeof(int),
                   cudaMemcpyHostToDevice);
        return fail(FDTD_ETIMEOUT, "a bounded device-side wait expired in the batched step");
    }
    return FDTD_OK;
}

int fdtd_batch_work_items(const fdtd_batch* b) { return b ? b->nitems : -1; }

void fdtd_batch_destroy(fdtd_batch* b)
{
    if (!b) return;
    for (int p = 0; p < 2; ++p)
        if (b->built[p]) cudaGraphExecDestroy(b->exec[p]);
    cudaStreamDestroy(b->capture);
    delete b;
}

}  // extern "C"
