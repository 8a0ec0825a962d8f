// Internal definitions shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "degrid.h"

namespace dg {

// Footprint of the paper's kernels (Section "Implementation"): G_uv has
// support 8 x 8, G_w support 4.  One warp covers one v-row of the footprint:
// lane = a * 4 + c holds the samples (a, c) of all 8 rows b.
constexpr int kUV = 8;
constexpr int kW = 4;
constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Subgrid shape and oversampling, passed by value to every kernel.
struct Geometry {
    int nx, ny, nz;
    int log2_uv_os;     // uv oversampling = 2^log2_uv_os
    int log2_w_os;      // w oversampling = 2^log2_w_os
    int row_stride;     // elements between rows y and y + 1: nx * nz
    int64_t plane;      // elements per subgrid: ny * nx * nz
};

// ---------------------------------------------------------------------------
// Coordinate step (Section "Implementation": start point g and GCF rows).
//
// p = rint(q * 2^k) with ties to even is computed exactly with integer
// operations on the IEEE-754 bit pattern of q, so no FP64 arithmetic is
// issued (FP64 throughput is low on this part).  With m the 53-bit
// significand and e the biased exponent, |q| * 2^k = m * 2^(e - 1075 + k).
// Returns false for non-finite q or |q * 2^k| >= 2^62.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool snap_rint(double q, int log2_os, long long &p)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(q);
    const int e = (int)((bits >> 52) & 0x7ff);
    if (e == 0x7ff)
        return false;                       // inf / nan
    const unsigned long long m = (bits & 0x000fffffffffffffull) | (e ? 0x0010000000000000ull : 0ull);
    const int shift = (e ? e : 1) - 1075 + log2_os;
    unsigned long long mag;
    if (shift >= 0) {
        if (shift > 9)
            return false;                   // |q * O| >= 2^62
        mag = m << shift;
    } else {
        const int r = -shift;
        if (r > 54) {
            mag = 0;                        // |q * O| < 0.25
        } else {
            const unsigned long long whole = m >> r;
            const unsigned long long rem = m & ((1ull << r) - 1ull);
            const unsigned long long half = 1ull << (r - 1);
            mag = whole + ((rem > half || (rem == half && (whole & 1ull))) ? 1ull : 0ull);
        }
    }
    p = (bits >> 63) ? -(long long)mag : (long long)mag;
    return true;
}

// One axis: start = floor(p / O) - W/2 + 1 and f = p mod O; valid when the
// footprint lies in [0, n).
__device__ __forceinline__ bool snap_axis(double q, int log2_os, int support, int n,
                                          int &start, int &frac)
{
    long long p;
    if (!snap_rint(q, log2_os, p))
        return false;
    const long long i = p >> log2_os;       // arithmetic shift = floor division
    frac = (int)(p & ((1ll << log2_os) - 1));
    const long long s = i - support / 2 + 1;
    start = (int)s;
    return s >= 0 && s <= (long long)(n - support);
}

struct VisCoords {
    int x0, y0, z0, fu, fv, fw;
};

__device__ __forceinline__ bool visibility_coords(double u, double v, double w,
                                                  const Geometry &g, VisCoords &c)
{
    const bool ok_u = snap_axis(u, g.log2_uv_os, kUV, g.nx, c.x0, c.fu);
    const bool ok_v = snap_axis(v, g.log2_uv_os, kUV, g.ny, c.y0, c.fv);
    const bool ok_w = snap_axis(w, g.log2_w_os, kW, g.nz, c.z0, c.fw);
    return ok_u && ok_v && ok_w;
}

// ---------------------------------------------------------------------------
// Subgrid storage types: every element becomes a float2 (re, im).
// ---------------------------------------------------------------------------
template <int DT> struct Storage;

template <> struct Storage<DG_C64> {
    static constexpr int kBytes = 8;
    __device__ __forceinline__ static float2 load(const void *base, int64_t i)
    {
        return __ldg(reinterpret_cast<const float2 *>(base) + i);
    }
};

template <> struct Storage<DG_C32_F16> {
    static constexpr int kBytes = 4;
    __device__ __forceinline__ static float2 load(const void *base, int64_t i)
    {
        const unsigned u = __ldg(reinterpret_cast<const unsigned *>(base) + i);
        __half2 h = *reinterpret_cast<const __half2 *>(&u);
        return __half22float2(h);
    }
};

template <> struct Storage<DG_C32_BF16> {
    static constexpr int kBytes = 4;
    __device__ __forceinline__ static float2 load(const void *base, int64_t i)
    {
        const unsigned u = __ldg(reinterpret_cast<const unsigned *>(base) + i);
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
};

// Status words kept by a plan on the device.
struct DeviceStatus {
    unsigned long long n_invalid;   // visibilities with an out-of-range footprint
    unsigned long long flags;       // kFlagOffsets, kFlagCapacity
};
constexpr unsigned long long kFlagOffsets = 1ull;
constexpr unsigned long long kFlagCapacity = 2ull;

// Work decomposition: chunk k covers visibilities
// [vis_offsets[s] + j * chunk, min(... + chunk, vis_offsets[s + 1])).
struct ChunkRef {
    int s;
    int j;
};

struct Schedule {
    const int64_t *vis_offsets;
    const ChunkRef *chunks;
    const int *n_chunks;            // device scalar written by the scheduler
    int *work_counter;              // zeroed before every launch
    int chunk;
};

// Launch helpers implemented in schedule.cu.
cudaError_t launch_schedule(cudaStream_t st, const int64_t *vis_offsets, int n_subgrids,
                            int64_t n_vis, int chunk, int *prefix, int *n_chunks,
                            ChunkRef *chunks, int capacity, int *work_counter,
                            DeviceStatus *status);

}  // namespace dg

// The plan object behind degrid_plan_t.
struct degrid_plan {
    int device;
    int sm_count;
    dg::Geometry geo;
    int uv_oversample, w_oversample;
    dg_dtype dtype;
    float *guv;                 // device FP32 [uv_os][8]
    float *gw;                  // device FP32 [w_os][4]
    dg::DeviceStatus *status;   // device
    int *work_counter;          // device [1]
    int *n_chunks;              // device [1]
    int *prefix;                // device [cap_subgrids + 1]
    dg::ChunkRef *chunks;       // device [cap_chunks]
    int cap_subgrids;
    int cap_chunks;
    int chunk;
    int warps_per_block;
    int blocks_per_sm;
    int max_blocks_degrid;      // occupancy results, 0 = not computed yet
    int max_blocks_adjoint;
    int n_slots;                // timing event pairs (0 = timing off)
    long long timed_launches;
    cudaEvent_t *ev_start, *ev_stop;
};

// Kernel launchers (one per translation unit).
cudaError_t dg_launch_degrid(degrid_plan *p, cudaStream_t st, const void *subgrids,
                             const float *scale, const double *uvw,
                             const int64_t *vis_offsets, float *vis_out, int grid_blocks);
cudaError_t dg_launch_adjoint(degrid_plan *p, cudaStream_t st, const double *uvw,
                              const int64_t *vis_offsets, const float *vis_in,
                              float *sub_out, int grid_blocks);
cudaError_t dg_launch_coords(degrid_plan *p, cudaStream_t st, const double *uvw,
                             int64_t n_vis, int32_t *coords_out);
int dg_max_blocks_per_sm_degrid(degrid_plan *p);
int dg_max_blocks_per_sm_adjoint(degrid_plan *p);
