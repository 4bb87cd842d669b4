// psc_tmap.cu -- tensor maps of the population buffers for the TMA staging of the pull
// (tma.cuh). Host code only: the driver's encoder is reached through the runtime's
// driver-entry-point query, so the library needs no link against the driver library.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#include "lattice.cuh"
#include "psc_internal.h"
#include "tma.cuh"

namespace psc {

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <class L, typename S>
static cudaError_t encode_t(CUtensorMap *map, CUtensorMapDataType dtype, const void *base, const Geom &g) {
    using B = TmaBox<L, S>;
    const cuuint64_t e = sizeof(S);
    if ((g.n[0] * e) % 16 != 0 || reinterpret_cast<uintptr_t>(base) % 16 != 0) return cudaErrorNotSupported;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t nx = g.n[0], ny = g.n[1], nz = g.n[2];
    cuuint64_t dims[4], strides[3];
    cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
    cuuint32_t rank;
    if (L::D == 2) {
        rank = 3;
        dims[0] = nx; dims[1] = ny; dims[2] = L::Q;
        strides[0] = nx * e; strides[1] = nx * ny * e;
        box[0] = B::BX; box[1] = L::TY; box[2] = 1;
    } else {
        rank = 4;
        dims[0] = nx; dims[1] = ny; dims[2] = nz; dims[3] = L::Q;
        strides[0] = nx * e; strides[1] = nx * ny * e; strides[2] = nx * ny * nz * e;
        box[0] = B::BX; box[1] = L::TY; box[2] = L::TZ; box[3] = 1;
    }
    for (cuuint32_t r = 0; r + 1 < rank; ++r)
        if (strides[r] >= (1ull << 40)) return cudaErrorNotSupported;
    const CUresult r = enc(map, dtype, rank, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorNotSupported;
}

cudaError_t encode_pop_tmap(CUtensorMap *map, int storage, int lattice, const void *base, const Geom &g) {
    const bool d2 = (lattice == 9);
    switch (storage) {
    case ST_F32:
        return d2 ? encode_t<D2Q9, float>(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, g)
                  : encode_t<D3Q19, float>(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, base, g);
    case ST_F16:
        return d2 ? encode_t<D2Q9, __half>(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, base, g)
                  : encode_t<D3Q19, __half>(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, base, g);
    case ST_BF16:
        return d2 ? encode_t<D2Q9, __nv_bfloat16>(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, g)
                  : encode_t<D3Q19, __nv_bfloat16>(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, base, g);
    default:
        return cudaErrorNotSupported;
    }
}

}  // namespace psc
