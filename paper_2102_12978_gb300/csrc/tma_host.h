// tma_host.h -- host helpers that encode the TMA tensor maps of a grid.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "grid_impl.h"

namespace fdtd {

inline PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 3-D tiled tensor map over one pitched [nz][ny][pitch] array; elements past
// nx / ny (and before 0) read as zero.
inline bool encode_map(CUtensorMap* m, void* base, size_t elem, const fdtd_grid_desc& d, int pitch, int bx,
                       int by)
{
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {cuuint64_t(d.nx), cuuint64_t(d.ny), cuuint64_t(d.nz)};
    cuuint64_t strides[2] = {cuuint64_t(pitch) * elem, cuuint64_t(pitch) * d.ny * elem};
    cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

inline int ty_slot(int ty) { return ty == 4 ? 0 : (ty == 8 ? 1 : 2); }

template <typename real, int TY>
inline bool tma_maps(fdtd_grid* g, int cur, TmaMaps** out)
{
    int sl = ty_slot(TY);
    if (!g->maps_ok[cur][sl]) {
        using T = TmaTile<real, TY>;
        char* A = static_cast<char*>(g->arena);
        TmaMaps& m = g->maps[cur][sl];
        bool ok = true;
        for (int c = 0; c < 3; ++c) {
            ok = ok && encode_map(&m.e[c], A + g->L.field[cur][c], sizeof(real), g->desc, g->L.pitch, T::BX, T::EBY);
            ok = ok && encode_map(&m.h[c], A + g->L.field[cur][3 + c], sizeof(real), g->desc, g->L.pitch, T::BX,
                                  T::HBY);
        }
        void* fbase = g->desc.fluence ? static_cast<void*>(A + g->L.fluence) : static_cast<void*>(A + g->L.field[cur][0]);
        ok = ok && encode_map(&m.f, fbase, 8, g->desc, g->L.pitch, T::FBX, T::FBY);
        if (!ok) return false;
        g->maps_ok[cur][sl] = true;
    }
    *out = &g->maps[cur][sl];
    return true;
}

}  // namespace fdtd
