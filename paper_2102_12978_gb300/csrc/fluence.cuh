// fluence.cuh -- the fluence reducer: turns the per-cell accumulator into a
// dense FP64 array, optionally scaled (scale = 1 / (window length) gives the
// intensity (1/tau) integral |S| dt of Section 5 over a window of whole periods).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fdtd {

__device__ __forceinline__ double flu_value(double v) { return v; }
__device__ __forceinline__ double flu_value(float2 v) { return double(v.x) - double(v.y); }

template <typename acc_t>
__global__ void fluence_export(const acc_t* __restrict__ F, double* __restrict__ out, int nx, int ny, int nz,
                               int pitch, double scale)
{
    const long long total = (long long)nx * ny * nz;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int i = int(q % nx);
        const long long r = q / nx;
        const int j = int(r % ny);
        const int k = int(r / ny);
        out[q] = scale * flu_value(F[((long long)k * ny + j) * pitch + i]);
    }
}

}  // namespace fdtd
