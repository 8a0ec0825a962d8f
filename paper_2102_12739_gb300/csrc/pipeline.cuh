// Batch pipeline shared by the degridding and gridding kernels.
//
// A persistent grid of warps claims chunks of consecutive visibilities of
// one subgrid (schedule.cu; claims pipelined one chunk ahead) and walks each
// chunk in batches of 32 visibilities (the gridding kernel) or steps of two
// such halves (the degridding kernel).  For every batch, lane i snaps
// visibility i (exact integer rint of its FP64 coordinates, internal.cuh),
// keeps its footprint key and w-kernel row in registers, and copies its g_u
// and g_v rows into the warp's shared-memory stage with cp.async; the small w
// table is kept in the CTA's shared memory.  The paper's D1 likewise computes
// the coordinates of all N_b visibilities of a block cooperatively into
// shared memory before the sums (Section "Implementation").
#pragma once

#include "internal.cuh"

namespace dg {
namespace {

constexpr int kBatch = 32;                  // visibilities per batch
constexpr int kUVRow = 8;                   // floats per uv table row (32 B)
constexpr int kWRow = 4;                    // floats per w table row (16 B)

// ---- PTX wrappers ---------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous global -> shared copy (L2 only), grouped per batch.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---- batch stream -----------------------------------------------------------

struct Batch {
    int s;          // subgrid
    int n;          // visibilities in this batch (1..kStep), 0 = none
    long long b0;   // first visibility
    long long end;  // end of the chunk
};

// Bulk prefetch of [p, p + bytes) into L2 (a hint: no completion, no data
// returned).  Only the 16-byte aligned interior of the range is requested,
// so nothing outside it is touched.
__device__ __forceinline__ void prefetch_l2(const void *p, long long bytes)
{
    const unsigned long long a = ((unsigned long long)p + 15ull) & ~15ull;
    const unsigned long long e = ((unsigned long long)p + (unsigned long long)bytes) & ~15ull;
    if (bytes > 0 && e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a)) : "memory");
}

// Per-visibility input streams of the chunk a warp will work on next: they
// are prefetched into L2 when its descriptor arrives, a whole chunk before
// the first load, so the loads of the batch pipeline find them in L2
// instead of waiting for HBM.
struct Prefetch {
    const void *a;      // stream 1 (or nullptr), a_bytes per visibility
    int a_bytes;
    const void *b;      // stream 2 (or nullptr)
    int b_bytes;
};

// Claims chunks with an atomic counter, one claim ahead: while a warp works
// on a chunk it already holds the descriptor of the next one, and the atomic
// for the one after that is in flight.  Batches of kStep visibilities.
template <int kStep>
struct ClaimerT {
    const Schedule &sched;
    Prefetch pf;
    int total;
    int lane;
    int pend;           // lane 0: atomic result not yet consumed
    ChunkDesc next;     // descriptor of the chunk after the current one
    int next_valid;

    __device__ void prefetch_next() const
    {
        if (lane == 0 && next_valid) {
            if (pf.a)
                prefetch_l2(static_cast<const char *>(pf.a) + next.lo * pf.a_bytes, (long long)next.n * pf.a_bytes);
            if (pf.b)
                prefetch_l2(static_cast<const char *>(pf.b) + next.lo * pf.b_bytes, (long long)next.n * pf.b_bytes);
        }
    }

    __device__ ClaimerT(const Schedule &sc, int lane_, Prefetch pf_ = Prefetch{nullptr, 0, nullptr, 0})
        : sched(sc), pf(pf_), lane(lane_)
    {
        total = *sc.n_chunks;
        int a = 0, b = 0;
        if (lane == 0) {
            a = atomicAdd(sc.work_counter, 1);
            b = atomicAdd(sc.work_counter, 1);
        }
        a = __shfl_sync(kFull, a, 0);
        pend = b;
        next_valid = a < total;
        if (next_valid)
            next = sc.chunks[a];
    }

    // Start the next claimed chunk; returns its first batch (n = 0 when done).
    __device__ Batch claim()
    {
        Batch bt{0, 0, 0, 0};
        if (!next_valid)
            return bt;
        const ChunkDesc cur = next;
        const int k = __shfl_sync(kFull, pend, 0);
        next_valid = k < total;
        if (next_valid)
            next = sched.chunks[k];
        prefetch_next();
        if (lane == 0)
            pend = atomicAdd(sched.work_counter, 1);
        bt.s = cur.s;
        bt.b0 = cur.lo;
        bt.end = cur.lo + cur.n;
        bt.n = (int)min((long long)kStep, bt.end - bt.b0);
        return bt;
    }

    __device__ Batch advance(const Batch &b)
    {
        if (b.n == 0)
            return b;
        Batch nb = b;
        nb.b0 = b.b0 + kStep;
        if (nb.b0 >= b.end)
            return claim();
        nb.n = (int)min((long long)kStep, b.end - nb.b0);
        return nb;
    }
};

using Claimer = ClaimerT<kBatch>;

// The visibilities [b0 + 32h, b0 + 32h + 32) of a batch of 64.
__device__ __forceinline__ Batch half_of(const Batch &b, int h)
{
    Batch r = b;
    r.b0 = b.b0 + kBatch * h;
    r.n = max(0, min(kBatch, b.n - kBatch * h));
    return r;
}

struct Coords3 {
    double u, v, w;
};

__device__ __forceinline__ Coords3 load_uvw(const double *__restrict__ uvw, const Batch &b, int lane)
{
    Coords3 c{0.0, 0.0, 0.0};
    if (lane < b.n) {
        const double *p = uvw + 3 * (b.b0 + lane);
        c.u = __ldg(p);
        c.v = __ldg(p + 1);
        c.w = __ldg(p + 2);
    }
    return c;
}

// Row stage: the g_u and g_v rows of 32 visibilities, 32 bytes per row.  The
// two 16-byte halves trade places on rows with bit 2 set, so that lanes
// reading the same half of 8 consecutive rows hit 8 different bank groups,
// while each row still fills one contiguous 32-byte slot (its two copies stay
// one L2 request).  (A 48-byte padded row stride also avoids the conflicts
// with fixed half offsets, but its larger footprint took L1 capacity from
// the coordinate loads and ran slower.)
struct alignas(128) RowStage {
    float4 u[kBatch][2];
    float4 v[kBatch][2];
    __device__ static int slot(int r, int h) { return h ^ ((r >> 2) & 1); }
};

// Slot of half `h` of row `r` in a RowStage row.
__device__ __forceinline__ int row_half(int r, int h) { return RowStage::slot(r, h); }

// What issue_rows leaves in registers for the summing step: this lane's
// visibility's footprint key (-1 when invalid or past the batch) and w row,
// whether the whole batch shares lane 0's key and row, and otherwise how
// many runs of equal key and row it holds.
struct Issued {
    int key, fw;
    int key0, fw0;
    bool uniform;
    int runs;           // runs of equal (key, w row) among the valid visibilities (1 if uniform)
    int blk;            // 2D G_uv table: weight block fv * O + fu of this visibility (0 if invalid)
};

// Stage 2 of a degridding batch: snap, and copy the g_u / g_v rows into the
// stage (2 lanes per 32-byte row, so each row is one request).
// With kRows = false (a 2D G_uv table, read by the summing lanes themselves)
// no rows are staged; the weight block index is kept instead.
template <class Stage, bool kRows = true>
__device__ __forceinline__ Issued issue_rows(const Batch &b, const Coords3 &c, const Geometry &g,
                                             Stage &S, const float *__restrict__ guv, int lane,
                                             DeviceStatus *status, bool commit = true)
{
    const bool in = lane < b.n;
    VisCoords vc;
    bool valid = in && visibility_coords(c.u, c.v, c.w, g, vc);
#ifdef DEGRID_BOUNDS_CHECK
    if (valid)
        valid = indices_in_bounds((vc.y0 * g.nx + vc.x0) * g.nz + vc.z0, vc.fu, vc.fv, vc.fw, g, status);
#endif
    Issued r;
    r.key = valid ? (vc.y0 * g.nx + vc.x0) * g.nz + vc.z0 : -1;
    r.fw = valid ? vc.fw : 0;
    const int fu = valid ? vc.fu : 0, fv = valid ? vc.fv : 0;
    r.key0 = __shfl_sync(kFull, r.key, 0);
    r.fw0 = __shfl_sync(kFull, r.fw, 0);
    // lanes past the end of the batch compute values nobody stores
    r.uniform = __all_sync(kFull, !in || (r.key == r.key0 && r.fw == r.fw0)) && r.key0 >= 0;
    r.runs = 1;
    if (!r.uniform) {
        const int kp = __shfl_up_sync(kFull, r.key, 1), fp = __shfl_up_sync(kFull, r.fw, 1);
        r.runs = __popc(__ballot_sync(kFull, r.key >= 0 && (lane == 0 || r.key != kp || r.fw != fp)));
    }
    const unsigned bad = __ballot_sync(kFull, in && !valid);
    if (lane == 0 && bad)
        atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
    r.blk = (fv << g.log2_uv_os) + fu;
    if (!kRows) {
        if (commit)
            cp_async_commit();
        return r;
    }
    const int half = lane & 1;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int row = (lane >> 1) + 16 * m;
        const int xu = __shfl_sync(kFull, fu, row);
        const int xv = __shfl_sync(kFull, fv, row);
        cp_async16(smem_u32(&S.u[row][Stage::slot(row, half)]), guv + (size_t)xu * kUVRow + 4 * half);
        cp_async16(smem_u32(&S.v[row][Stage::slot(row, half)]), guv + (size_t)xv * kUVRow + 4 * half);
    }
    if (commit)
        cp_async_commit();
    return r;
}

// The w table ahead of the per-warp areas in dynamic shared memory.
__device__ __forceinline__ int wtable_bytes(const Geometry &g)
{
    return g.w_table_rows > 0 ? ((g.w_table_rows * kWRow * 4 + 127) & ~127) : 0;
}

// Copies the w table into shared memory (whole CTA); returns it, or nullptr
// when the table is too large and rows are fetched per batch instead.
__device__ __forceinline__ const float4 *load_wtable(const Geometry &g, const float *gwt,
                                                    unsigned char *smem)
{
    if (g.w_table_rows <= 0)
        return nullptr;
    float4 *t = reinterpret_cast<float4 *>(smem);
    const float4 *src = reinterpret_cast<const float4 *>(gwt);
    for (int i = threadIdx.x; i < g.w_table_rows; i += blockDim.x)
        t[i] = __ldg(src + i);
    __syncthreads();
    return t;
}

inline size_t wtable_bytes_host(const Geometry &g)
{
    return g.w_table_rows > 0 ? ((size_t)g.w_table_rows * kWRow * 4 + 127) & ~(size_t)127 : 0;
}

}  // namespace
}  // namespace dg
