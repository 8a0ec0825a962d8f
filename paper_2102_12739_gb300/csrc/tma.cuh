// TMA and mbarrier helpers of the kernels that move whole footprints between
// the stack and shared memory (the gather kernel reads them, the scattered
// gridding kernel adds them back).
//
// With nz = 4 a footprint row (8 columns x 4 samples) is one contiguous
// piece of the stack: 256 bytes in complex64, 128 in FP16/BF16 code pairs.
// The stack is described to the copy engine as a 2D tensor [S * ny rows]
// [nx * nz elements] and a footprint is one box of 8 rows x kBoxX elements,
// the row plus 16 bytes: row b of the box lands 16 b bytes past a 128-byte
// boundary, so 8 lanes reading the same column of the 8 rows hit 8 different
// bank groups (the extra 16 bytes are the next column's first samples, or
// zeros past the edge of the stack).  The box's x coordinate is x0 * nz, so
// x times the element size is a multiple of 16 bytes, as the copy requires.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"

namespace dg {
namespace {

template <int DT>
struct FootprintBox {
    static constexpr int kRowBytes = kUV * kW * Storage<DT>::kBytes;     // one footprint row: 256 / 128
    static constexpr int kPitch = kRowBytes + 16;                        // box row in shared memory
    static constexpr int kBoxX = kPitch / Storage<DT>::kBytes;           // box width, elements: 34 / 36
    static constexpr int kBytes = kUV * kPitch;                          // one box: 2176 / 1152
};

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// One arrival that also announces `bytes` of transfers for the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Waits for phase `parity` of the mbarrier, polling at most `limit` times;
// returns false (on every lane) when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, unsigned parity, int limit = kSpinLimit)
{
    bool ok = false;
    for (int i = 0; i < limit && !ok; ++i)
        ok = mbar_try_wait(bar, parity);
    return __all_sync(kFull, ok);
}

// TMA tensor copy of the box at (x, y) of the 2D tensor map into shared
// memory (128-byte aligned), completing as transfer bytes on the mbarrier.
__device__ __forceinline__ void tensor_copy_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbarrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// A 2D tensor map (host side): dim0 x dim1 elements of type `type`, rows
// `stride` bytes apart, boxes of box0 x box1 elements, no swizzle.
inline cudaError_t encode_2d(CUtensorMap *map, void *base, CUtensorMapDataType type, uint64_t dim0,
                             uint64_t dim1, uint64_t stride, uint32_t box0, uint32_t box1)
{
    // looked up once (a function-local static: initialised once, also under
    // concurrent first calls from several host threads)
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                               cudaEnableDefault, &q);
        return e == cudaSuccess && q == cudaDriverEntryPointSuccess
                   ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)
                   : nullptr;
    }();
    if (!encode)
        return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)dim0, (cuuint64_t)dim1};
    const cuuint64_t strides[1] = {(cuuint64_t)stride};
    const cuuint32_t box[2] = {(cuuint32_t)box0, (cuuint32_t)box1};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, type, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The tensor map of a stack of n_subgrids subgrids (host side), with boxes
// of 8 rows x box_x elements (FootprintBox<DT>::kBoxX for padded rows, or
// 32 for the bare footprint).
template <int DT>
cudaError_t encode_footprint_map(const degrid_plan *p, const void *subgrids, int n_subgrids, CUtensorMap *map,
                                 int box_x = FootprintBox<DT>::kBoxX)
{
    return encode_2d(map, const_cast<void *>(subgrids),
                     DT == DG_C64 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                     (uint64_t)p->geo.row_stride, (uint64_t)n_subgrids * p->geo.ny,
                     (uint64_t)p->geo.row_stride * Storage<DT>::kBytes, (uint32_t)box_x, (uint32_t)kUV);
}

}  // namespace
}  // namespace dg
