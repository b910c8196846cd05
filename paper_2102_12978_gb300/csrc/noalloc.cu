// noalloc.cu -- fluence read-out for callers that cannot allocate device memory.
//
// fdtd_fluence stages the exported fluence in a buffer of the grid's arena
// before copying it out.  Some callers cannot call cudaMalloc at all: code
// that runs while a caching allocator is not allowed to grow, inside hooks
// that must not allocate, or on systems where device memory is reserved up
// front.  fdtd_fluence_noalloc gives them the same result with the staging
// buffer in a file-scope device array of fixed size instead, and calls no
// allocating routine.
//
// The array belongs to this file's module.  Under CUDA's lazy module loading
// a module's globals become resident on a device only when the module is first
// used there, and that load allocates.  So the array's device address is
// looked up in fdtd_create_grid (noalloc_prepare), where allocating is
// allowed: from the first grid created on a device on, the array is resident
// there, and the read-out itself only reads the cached address.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "../../include/fdtd.h"
#include "fluence.cuh"
#include "grid_impl.h"

namespace fdtd {

// Staging area of the export: 16 MiB (2^21 doubles) per device, resident from
// the first fdtd_create_grid on that device until the process exits.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of the array per device (the array's name in host code is
// only a host-side handle, not a device address).  Written under the mutex
// by every grid creation on the device, so that a grid created after a
// cudaDeviceReset refreshes it; read without the lock by the read-out.
constexpr int kMaxDevices = 64;
static std::atomic<double*> g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mutex;

fdtd_status noalloc_prepare(int device)
{
    if (device < 0 || device >= kMaxDevices)
        return fail(FDTD_EINVAL, "device %d beyond the %d the library supports", device, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    void* p = nullptr;
    fdtd_status st = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "no-allocation scratch address");
    if (st != FDTD_OK) return st;
    g_scratch_ptr[device].store(static_cast<double*>(p), std::memory_order_release);
    return FDTD_OK;
}

}  // namespace fdtd

using namespace fdtd;

extern "C" {

size_t fdtd_fluence_noalloc_max_cells(void) { return kNoAllocScratchDoubles; }

fdtd_status fdtd_fluence_noalloc(fdtd_grid* g, void* dst, int on_device, int reset)
{
    if (!g || !dst) return fail(FDTD_EINVAL, "null argument");
    if (!g->desc.fluence) return fail(FDTD_ESTATE, "grid created without a fluence accumulator");
    const fdtd_status dev_st = check_device(g, "fdtd_fluence_noalloc");
    if (dev_st != FDTD_OK) return dev_st;
    const fdtd_grid_desc& d = g->desc;
    const size_t cells = size_t(d.nx) * d.ny * d.nz;
    if (cells > kNoAllocScratchDoubles)
        return fail(FDTD_EINVAL, "grid of %zu cells exceeds the %zu-cell limit of fdtd_fluence_noalloc", cells,
                    kNoAllocScratchDoubles);
    double* scratch = (g->device >= 0 && g->device < kMaxDevices)
                          ? g_scratch_ptr[g->device].load(std::memory_order_acquire)
                          : nullptr;
    if (!scratch) return fail(FDTD_ESTATE, "no staging array on device %d", g->device);
    char* A = static_cast<char*>(g->arena);
    const int blocks = 4 * (g->sm_count > 0 ? g->sm_count : 152);
    if (d.precision == FDTD_F64)
        fluence_export<double><<<blocks, 256, 0, g->stream>>>(reinterpret_cast<const double*>(A + g->L.fluence),
                                                              scratch, d.nx, d.ny, d.nz, g->L.pitch, 1.0);
    else
        fluence_export<float2><<<blocks, 256, 0, g->stream>>>(reinterpret_cast<const float2*>(A + g->L.fluence),
                                                               scratch, d.nx, d.ny, d.nz, g->L.pitch, 1.0);
    fdtd_status st = cuda_check(cudaGetLastError(), "fluence_export launch");
    if (st == FDTD_OK)
        st = cuda_check(cudaMemcpyAsync(dst, scratch, cells * 8,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream),
                        "copy fluence");
    if (st == FDTD_OK && reset)
        st = cuda_check(cudaMemsetAsync(A + g->L.fluence, 0, g->L.field_elems * 8, g->stream), "reset fluence");
    if (st != FDTD_OK) return st;
    return fdtd_sync(g);
}

}  // extern "C"
