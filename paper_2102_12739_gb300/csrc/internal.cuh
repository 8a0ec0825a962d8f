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
constexpr int kMaxDevices = 64;     // devices whose per-kernel launch attributes are cached

// Subgrid shape and oversampling, passed by value to every kernel.
struct Geometry {
    int nx, ny, nz;
    int log2_uv_os;     // uv oversampling = 2^log2_uv_os
    int log2_w_os;      // w oversampling = 2^log2_w_os
    int row_stride;     // elements between rows y and y + 1: nx * nz
    int64_t plane;      // elements per subgrid: ny * nx * nz
    int w_table_rows;   // w oversampling if the w table is staged in shared memory, else 0
};

// ---------------------------------------------------------------------------
// Coordinate step (Section "Implementation": start point g and GCF rows).
//
// Per axis with support W and oversampling O = 2^k: p = rint(q * O) with
// ties to even, i = floor(p / O), f = p - i * O, start = i - W/2 + 1; valid
// when 0 <= start <= n - W.  Computed exactly with one FP64 operation per
// axis (FP64 runs at a small fraction of the FP32 rate on this part, so no
// FP64 multiply or floor): q * 2^k is formed by adding k to the exponent
// field of q's high word (an integer add), and one conversion to a 32-bit
// integer rounds it to nearest, ties to even (cvt.rni: out-of-range values
// saturate, NaN converts to 0).  The rest is integer: f = p & (O - 1),
// i = p >> k (arithmetic, so floor for negative p).  Every input that is not
// a valid coordinate lands on an invalid start with no extra test:
//   * q = +-0 or denormal: the exponent add gives a number below 2^(k-1022),
//     p = 0, start < 0 (W >= 4);
//   * q < 0: p <= 0, start < 0;
//   * q * O >= 2^31 or q huge: p saturates at 2^31 - 1, start > n - W (the
//     plan requires n * O <= 2^31);
//   * inf, NaN, or an exponent that the add carries into the sign bit: the
//     pattern becomes a tiny negative number (p = 0), inf / NaN (p saturates
//     or is 0), all invalid as above.
// Checked against the exact definition on the CPU (every special value,
// exact ties and their neighbours, random bit patterns) and on the GPU by the
// coordinate tests.  A form with 32-bit integer funnel shifts on the FP64
// bit pattern (no FP64 operation at all) took 17 integer instructions per
// axis against 5 here and measured 1% slower in the degridding kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool snap_axis(double q, int log2_os, int support, int n,
                                          int &start, int &frac)
{
    const unsigned hi = (unsigned)__double2hiint(q) + ((unsigned)log2_os << 20);
    const int p = __double2int_rn(__hiloint2double((int)hi, __double2loint(q)));
    frac = p & ((1 << log2_os) - 1);
    start = (p >> log2_os) - (support / 2 - 1);
    return (unsigned)start <= (unsigned)(n - support);
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

// load4(base, i): elements i .. i + 3 with 16-byte loads; i must be a
// multiple of kQuad and the base 16-byte aligned (the launcher checks both
// and passes the result to the kernels).
template <> struct Storage<DG_C64> {
    static constexpr int kBytes = 8;
    static constexpr int kQuad = 2;     // elements per 16 bytes
    __device__ __forceinline__ static float2 load(const void *base, int64_t i)
    {
        return __ldg(reinterpret_cast<const float2 *>(base) + i);
    }
    __device__ __forceinline__ static void load4(const void *base, int64_t i, float2 (&s)[4])
    {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(base) + (i >> 1));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(base) + (i >> 1) + 1);
        s[0] = make_float2(a.x, a.y);
        s[1] = make_float2(a.z, a.w);
        s[2] = make_float2(b.x, b.y);
        s[3] = make_float2(b.z, b.w);
    }
};

template <> struct Storage<DG_C32_F16> {
    static constexpr int kBytes = 4;
    static constexpr int kQuad = 4;
    __device__ __forceinline__ static float2 cvt(unsigned u)
    {
        __half2 h = *reinterpret_cast<const __half2 *>(&u);
        return __half22float2(h);
    }
    __device__ __forceinline__ static float2 load(const void *base, int64_t i)
    {
        return cvt(__ldg(reinterpret_cast<const unsigned *>(base) + i));
    }
    __device__ __forceinline__ static void load4(const void *base, int64_t i, float2 (&s)[4])
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(base) + (i >> 2));
        s[0] = cvt(q.x);
        s[1] = cvt(q.y);
        s[2] = cvt(q.z);
        s[3] = cvt(q.w);
    }
};

template <> struct Storage<DG_C32_BF16> {
    static constexpr int kBytes = 4;
    static constexpr int kQuad = 4;
    __device__ __forceinline__ static float2 cvt(unsigned u)
    {
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
    __device__ __forceinline__ static float2 load(const void *base, int64_t i)
    {
        return cvt(__ldg(reinterpret_cast<const unsigned *>(base) + i));
    }
    __device__ __forceinline__ static void load4(const void *base, int64_t i, float2 (&s)[4])
    {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(base) + (i >> 2));
        s[0] = cvt(q.x);
        s[1] = cvt(q.y);
        s[2] = cvt(q.z);
        s[3] = cvt(q.w);
    }
};

// Status words kept by a plan on the device.
struct DeviceStatus {
    unsigned long long n_invalid;   // visibilities with an out-of-range footprint
    unsigned long long flags;       // kFlagOffsets, kFlagCapacity
};
constexpr unsigned long long kFlagOffsets = 1ull;
constexpr unsigned long long kFlagCapacity = 2ull;
constexpr unsigned long long kFlagTimeout = 4ull;   // a bounded device wait gave up
constexpr unsigned long long kFlagBounds = 8ull;    // an index check failed (DEGRID_BOUNDS_CHECK builds)

#ifdef DEGRID_BOUNDS_CHECK
// Index checks of the bounds-checking build: every index the coordinate step
// produces for a valid visibility against the extents of what it addresses.
// A failure records kFlagBounds; the caller then treats the visibility as
// invalid, so nothing is read or written through the bad index.
__device__ __forceinline__ bool indices_in_bounds(int key, int fu, int fv, int fw, const Geometry &g,
                                                  DeviceStatus *status)
{
    const int64_t last = (int64_t)key + (int64_t)(kUV - 1) * g.row_stride + (int64_t)(kUV - 1) * g.nz + (kW - 1);
    const bool ok = key >= 0 && last < g.plane && (unsigned)fu < (1u << g.log2_uv_os) &&
                    (unsigned)fv < (1u << g.log2_uv_os) && (unsigned)fw < (1u << g.log2_w_os);
    if (!ok)
        atomicOr(&status->flags, kFlagBounds);
    return ok;
}
#endif

// Work decomposition: chunk k covers the n visibilities [lo, lo + n) of
// subgrid s (n <= chunk size; a chunk never straddles two subgrids).
struct alignas(16) ChunkDesc {
    int s;
    int n;
    long long lo;
};

struct Schedule {
    const ChunkDesc *chunks;
    const int *n_chunks;            // device scalar written by the scheduler
    int *work_counter;              // zeroed by the scheduler before every launch
};

// Bound on the polls of any device-side wait (mbarrier phase); a wait that
// exceeds it records kFlagTimeout and the warp stops working.
constexpr int kSpinLimit = 1 << 22;

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The kernels of one call run back to back on
// a stream (scan -> chunk table -> sums); each later one is launched with
// programmatic stream serialisation, so it is scheduled while its
// predecessor still runs and does its independent setup (w table, barriers)
// meanwhile.  pdl_wait() returns once the predecessor grid has completed and
// its writes are visible: every kernel calls it before it reads or writes
// anything its predecessor (or the work before that) touches.
// pdl_trigger() lets the successor be scheduled early.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches `kernel` so that it may overlap the tail of the previous kernel
// in the stream (it must call pdl_wait() before touching shared data).
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

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
    float *guv2;                // device FP32 [uv_os][uv_os][8][8] for a 2D G_uv table, else nullptr
    dg::DeviceStatus *status;   // device
    int *work_counter;          // device [1]
    int *n_chunks;              // device [1]
    int *prefix;                // device [cap_subgrids + 1]
    dg::ChunkDesc *chunks;      // device [cap_chunks]
    int cap_subgrids;
    int cap_chunks;
    int chunk;
    int warps_per_block;
    int blocks_per_sm;
    int compensated;            // compensated (TwoSum) reduction of the lane partials
    int direct_runs;            // non-uniform halves with at least this many runs take the direct sum
    int gather;                 // sum through the gather kernel (gather.cu)
    int host_direct;            // degrid_execute_host reads page-locked host inputs in place
    int host_inputs;            // set during such a call: the kernel's inputs are in host memory
    int max_blocks_degrid;      // occupancy results, 0 = not computed yet
    int max_blocks_adjoint;
    struct dg_host_exec *hostx; // streams and staging of degrid_execute_host (host_exec.cu), lazily
    int n_slots;                // timing event pairs (0 = timing off)
    long long timed_launches;
    cudaEvent_t *ev_start, *ev_stop;
};

void dg_free_host_exec(degrid_plan *p);   // host_exec.cu

#include <atomic>
#include <mutex>

// Dynamic shared memory of a kernel instance beyond the default limit
// (cudaFuncSetAttribute, per device).  `rec` (one per instance and device)
// holds the largest size opened so far and the attribute only grows, so the
// launches and occupancy queries of plans of different sizes, also from
// several host threads, never find it below what they asked for.
template <class F>
cudaError_t dg_open_smem(std::atomic<size_t> &rec, F *func, size_t smem)
{
    if (rec.load(std::memory_order_acquire) >= smem)
        return cudaSuccess;
    static std::mutex m;
    std::lock_guard<std::mutex> lock(m);
    if (rec.load(std::memory_order_relaxed) >= smem)
        return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        rec.store(smem, std::memory_order_release);
    return e;
}

// The record of device `device` in a per-instance table (devices past the
// table share a scratch record that never skips the call).
inline std::atomic<size_t> &dg_smem_record(std::atomic<size_t> (&table)[dg::kMaxDevices], int device)
{
    static thread_local std::atomic<size_t> scratch;
    if (device >= 0 && device < dg::kMaxDevices)
        return table[device];
    scratch.store(0);
    return scratch;
}

#include <nvtx3/nvToolsExt.h>

// An NVTX range over an entry point (plan creation, the execute calls), so
// profilers show the library's calls around its kernels; free when no tool
// is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


namespace dg {
// A list of fewer than kSparseItems * chunk visibilities is sparse (schedule.cu).
constexpr int kSparseItems = 64;

// The chunk table of a call (schedule.cu): items of `chunk` visibilities,
// or with `small` > 0 sparse lists first in items of `small` (capacity from
// dg_schedule_capacity).
cudaError_t launch_schedule(cudaStream_t st, const int64_t *vis_offsets, int n_subgrids,
                            int64_t n_vis, int chunk, int small, int *prefix, int *n_chunks,
                            ChunkDesc *chunks, int capacity, int *work_counter,
                            DeviceStatus *status);
}  // namespace dg

// Items per call that the chunk table must hold: lists are cut into items
// of `chunk`, sparse lists (fewer than kSparseItems * chunk visibilities)
// into items of `small` (if > 0), each list ending in one partial item.
inline int64_t dg_schedule_capacity(int S, int64_t n_vis, int chunk, int small)
{
    int64_t need = n_vis / chunk + S + 1;
    if (small > 0) {
        const int64_t sparse = n_vis / small + S;
        const int64_t bound = (int64_t)S * (dg::kSparseItems * (int64_t)chunk / small + 1);
        need += sparse < bound ? sparse : bound;
    }
    return need;
}

// Item size of the sparse lists in the allocating entry points (0: the
// fixed-scratch entry point keeps one item size).
inline int dg_small_items(int chunk) { return chunk > 64 ? 64 : 0; }

// Kernel launchers (one per translation unit).
cudaError_t dg_launch_degrid(degrid_plan *p, cudaStream_t st, const void *subgrids,
                             const float *scale, const double *uvw,
                             const int64_t *vis_offsets, float *vis_out, int grid_blocks);
cudaError_t dg_launch_adjoint(degrid_plan *p, cudaStream_t st, const double *uvw,
                              const int64_t *vis_offsets, const float *vis_in,
                              float *sub_out, int grid_blocks);
cudaError_t dg_launch_coords(degrid_plan *p, cudaStream_t st, const double *uvw,
                             int64_t n_vis, int32_t *coords_out);
cudaError_t dg_launch_gather(degrid_plan *p, cudaStream_t st, const void *subgrids, int n_subgrids,
                             const float *scale, const double *uvw, float *vis_out, int grid_blocks);
int dg_gather_warps(dg_dtype dtype);            // warps per CTA of the gather kernel
cudaError_t dg_launch_scatter(degrid_plan *p, cudaStream_t st, int n_subgrids, const double *uvw,
                              const float *vis_in, float *sub_out, int grid_blocks);
int dg_scatter_warps();                         // warps per CTA of the scattered gridding kernel
bool dg_gather_supported(const degrid_plan *p);
int dg_max_blocks_per_sm_degrid(degrid_plan *p);
int dg_max_warps_per_block();        // largest warps_per_block the kernels are built for
int dg_max_blocks_per_sm_adjoint(degrid_plan *p);
