// peak.cu -- measured FP64 fused multiply-add rate of the device: the
// denominator of the FP64 passes' roofline.  GB300's FP64 pipe is a small
// fraction of its FP32 rate, and the FP64 cell passes (one FP64 FMA or add
// per operation of Section 4's update and of the Section 2 fluence) run into
// that pipe before HBM.  The paper has no counterpart.  Also the device
// norm of the FP64 fluence term on an array, for its accuracy test.
#include <cuda_runtime.h>

#include "../../include/fdtd.h"
#include "grid_impl.h"

namespace fdtd {

// CHAINS independent FMA chains per thread, `iters` FMAs each.  The chains
// converge to c / (1 - b) for 0 < b < 1, so they stay finite and normal; the
// sum is stored only if it equals a value it cannot reach, which keeps every
// FMA live without a store per thread.
template <int CHAINS>
__global__ void fp64_fma_rate(double* sink, int iters, double b, double c)
{
    double acc[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc[k] = 1e-3 * threadIdx.x + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) acc[k] = fma(acc[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += acc[k];
    if (s == -1.0) sink[0] = s;
}

template <int CHAINS>
static cudaError_t time_fma(double* sink, cudaStream_t s, int blocks, int iters, float* ms)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
    fp64_fma_rate<CHAINS><<<blocks, 256, 0, s>>>(sink, 64, 0.999999, 1e-6);   // warm-up
    cudaEventRecord(e0, s);
    fp64_fma_rate<CHAINS><<<blocks, 256, 0, s>>>(sink, iters, 0.999999, 1e-6);
    cudaEventRecord(e1, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

__global__ void vec_norm_array(const double* __restrict__ x, double* __restrict__ out, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = vec_norm(x[i]);
}

}  // namespace fdtd

using namespace fdtd;

extern "C" {

fdtd_status fdtd_measure_fp64_rate(void* dev_sink, void* stream, int chains, int iters, double* fma_per_s,
                                   double* ms)
{
    if (!dev_sink || !fma_per_s || !ms || iters < 1 || (chains != 1 && chains != 8))
        return fail(FDTD_EINVAL, "fdtd_measure_fp64_rate: invalid argument");
    int dev = 0, sms = 0;
    fdtd_status st = cuda_check(cudaGetDevice(&dev), "current device");
    if (st == FDTD_OK)
        st = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (st != FDTD_OK) return st;
    const int blocks = 8 * sms;   // 2048 threads per SM
    float t = 0.0f;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* sink = static_cast<double*>(dev_sink);
    const cudaError_t e = chains == 8 ? time_fma<8>(sink, s, blocks, iters, &t) : time_fma<1>(sink, s, blocks, iters, &t);
    st = cuda_check(e, "FP64 FMA rate kernel");
    if (st != FDTD_OK) return st;
    *ms = t;
    *fma_per_s = double(blocks) * 256.0 * double(iters) * chains / (t * 1e-3);
    return FDTD_OK;
}

fdtd_status fdtd_debug_vec_norm(const void* dev_x, void* dev_out, int64_t n, void* stream)
{
    if (n < 0) return fail(FDTD_EINVAL, "fdtd_debug_vec_norm: n < 0");
    if (n == 0) return FDTD_OK;
    if (!dev_x || !dev_out) return fail(FDTD_EINVAL, "fdtd_debug_vec_norm: null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long blocks = (n + 255) / 256;
    if (blocks > 0x7fffffffLL) return fail(FDTD_EINVAL, "fdtd_debug_vec_norm: n too large");
    vec_norm_array<<<unsigned(blocks), 256, 0, s>>>(static_cast<const double*>(dev_x), static_cast<double*>(dev_out),
                                                    n);
    fdtd_status st = cuda_check(cudaGetLastError(), "vec_norm kernel");
    if (st == FDTD_OK) st = cuda_check(cudaStreamSynchronize(s), "vec_norm kernel");
    return st;
}

}  // extern "C"
