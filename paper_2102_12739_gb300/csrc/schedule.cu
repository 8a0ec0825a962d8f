// Work decomposition for the persistent kernels.
//
// The paper launches a grid of max_S(N_vis,S / N_b) x S thread blocks
// (Eq. 1) and notes that uneven visibility counts leave most of it idle.
// Here the visibilities of every subgrid are cut into work items (an item
// never straddles two subgrids): sparse lists into items of `small`
// visibilities at the front of the table, the others into items of
// `chunk` after them (list_items below).  A persistent grid claims the items
// in table order with an atomic counter, so the load is balanced whatever
// the counts are, and the expensive sparse items are done first.
//
// The chunk table is built on the device, so no host synchronisation is
// needed and the whole call can be captured in a CUDA graph.  For up to
// kSchedMaxS subgrids one kernel does it: every block scans the item counts
// of all subgrids into the starts in its shared memory (the scan is small
// and every block gets the same result), block 0 also validates vis_offsets
// and resets the work counter, and each block writes the descriptors
// (s, count, first visibility) of its share of the subgrids.  Larger stacks
// take two kernels: chunk_prefix (one block scans into prefix[S + 1] in
// global memory) and chunk_fill (the descriptors).
#include "internal.cuh"

namespace dg {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kSchedMaxS = 4096;            // subgrids the one-kernel schedule scans in shared memory
constexpr int kSchedMaxBlocks = 1024;
constexpr int kSchedThreads = 256;          // the one-kernel schedule's blocks

// Work items of subgrid s.  Lists of fewer than kSparseItems * chunk
// visibilities are sparse: their consecutive visibilities rarely share a
// footprint, so each of them costs many times a dense one (one M build per
// visibility or so).  With `small` > 0 such a list is cut into items of
// `small` visibilities and its items go to the front of the table, so they
// are claimed first and the end of a call is left to cheap dense items
// (otherwise one sparse item claimed last can hold its warp long after the
// others are done).  With `small` = 0 every list is dense: items of `chunk`
// in subgrid order.

struct ListItems {
    int size;           // visibilities per item
    bool sparse;        // items at the front of the table
    long long count;    // items of the list
};

__device__ __forceinline__ ListItems list_items(long long len, int chunk, int small)
{
    ListItems r;
    r.sparse = small > 0 && len < (long long)kSparseItems * chunk;
    r.size = r.sparse ? small : chunk;
    r.count = (len + r.size - 1) / r.size;
    return r;
}

// Block-wide inclusive scan of a pair (x.x, x.y) over threads; every thread
// gets its inclusive pair, and `tot` (shared) the block total.
__device__ __forceinline__ longlong2 block_scan2(longlong2 x, longlong2 *warp_sums, longlong2 &tot)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x / kWarp;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long a = __shfl_up_sync(kFull, x.x, d), b = __shfl_up_sync(kFull, x.y, d);
        if (lane >= d) {
            x.x += a;
            x.y += b;
        }
    }
    if (lane == 31)
        warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        longlong2 t = lane < nw ? warp_sums[lane] : make_longlong2(0, 0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long a = __shfl_up_sync(kFull, t.x, d), b = __shfl_up_sync(kFull, t.y, d);
            if (lane >= d) {
                t.x += a;
                t.y += b;
            }
        }
        if (lane < nw)
            warp_sums[lane] = t;        // inclusive over warps
        if (lane == nw - 1)
            tot = t;
    }
    __syncthreads();
    if (wid > 0) {
        x.x += warp_sums[wid - 1].x;
        x.y += warp_sums[wid - 1].y;
    }
    return x;
}

// Start of every subgrid's items in the table into pre[0..S) (shared or
// global memory; sparse lists first, each part in subgrid order), each start
// clamped to `capacity`, and the (clamped) item total into pre[S]; every
// thread of the block gets the total.  With `lead` the block records
// malformed offsets and an overflowing total in the status flags.
__device__ long long scan_chunks(const int64_t *__restrict__ offs, int S, int64_t n_vis, int chunk, int small,
                                 int *pre, int capacity, bool lead, DeviceStatus *status)
{
    __shared__ longlong2 warp_sums[kScanThreads / kWarp];
    __shared__ longlong2 tot;
    __shared__ long long carry_sp, carry_dn, sparse_total;
    const int tid = threadIdx.x;
    const int nt = blockDim.x;              // a multiple of 32, at most kScanThreads
    if (tid == 0) {
        carry_sp = carry_dn = 0;
        if (lead && (offs[0] != 0 || offs[S] != n_vis))
            atomicOr(&status->flags, kFlagOffsets);
    }
    // pass 0 (only with small > 0) totals the sparse lists' items; pass 1
    // scans the (sparse, dense) item counts and writes each list's start: a
    // sparse list after the sparse items before it, a dense one after all
    // sparse items and the dense items before it
    long long sp_total = 0;
    for (int pass = small > 0 ? 0 : 1; pass < 2; ++pass) {
        __syncthreads();
        for (int base = 0; base < S; base += nt) {
            const int s = base + tid;
            longlong2 cnt = make_longlong2(0, 0);       // (sparse items, dense items)
            if (s < S) {
                const int64_t lo = offs[s], hi = offs[s + 1];
                if (lo >= 0 && lo <= hi && hi <= n_vis) {
                    const ListItems it = list_items(hi - lo, chunk, small);
                    (it.sparse ? cnt.x : cnt.y) = it.count;
                } else if (lead && pass == 1) {
                    atomicOr(&status->flags, kFlagOffsets);
                }
            }
            const longlong2 inc = block_scan2(cnt, warp_sums, tot);
            if (pass == 1 && s < S) {
                const long long start = cnt.x ? carry_sp + inc.x - cnt.x
                                              : sp_total + carry_dn + inc.y - cnt.y;
                pre[s] = (int)min(start, (long long)capacity);
            }
            __syncthreads();
            if (tid == 0) {
                carry_sp += tot.x;
                carry_dn += tot.y;
            }
            __syncthreads();
        }
        if (pass == 0) {
            if (tid == 0) {
                sparse_total = carry_sp;
                carry_sp = carry_dn = 0;
            }
            __syncthreads();
            sp_total = sparse_total;
        }
    }
    long long total = carry_sp + carry_dn;
    if (total > capacity) {
        if (lead && tid == 0)
            atomicOr(&status->flags, kFlagCapacity);
        total = capacity;
    }
    if (tid == 0)
        pre[S] = (int)total;
    __syncthreads();
    return total;
}

// Descriptors of the items of subgrids s = first, first + step, ...
__device__ __forceinline__ void fill_chunks(const int *pre, const int64_t *__restrict__ offs, int S,
                                            int64_t n_vis, int chunk, int small, int capacity,
                                            ChunkDesc *__restrict__ chunks, int first, int step)
{
    for (int s = first; s < S; s += step) {
        const int64_t vis_lo = offs[s], vis_hi = offs[s + 1];
        if (!(vis_lo >= 0 && vis_lo <= vis_hi && vis_hi <= n_vis))
            continue;                       // malformed (the scan gave it no items): none
        const ListItems it = list_items(vis_hi - vis_lo, chunk, small);
        const int lo = pre[s];
        const int hi = (int)min((long long)lo + it.count, (long long)capacity);
        for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
            const int64_t first_vis = vis_lo + (int64_t)(k - lo) * it.size;
            const int64_t last = min(first_vis + (int64_t)it.size, vis_hi);
            chunks[k] = ChunkDesc{s, (int)(last - first_vis), (long long)first_vis};
        }
    }
}

__global__ void __launch_bounds__(kSchedThreads)
chunk_schedule(const int64_t *__restrict__ offs, int S, int64_t n_vis, int chunk, int small,
               int *__restrict__ n_chunks, int capacity, int *__restrict__ work_counter,
               DeviceStatus *__restrict__ status, ChunkDesc *__restrict__ chunks)
{
    __shared__ int pre[kSchedMaxS + 1];
    pdl_trigger();                          // the summing kernel may be scheduled now
    const bool lead = blockIdx.x == 0;
    const long long total = scan_chunks(offs, S, n_vis, chunk, small, pre, capacity, lead, status);
    if (lead && threadIdx.x == 0) {
        *work_counter = 0;
        *n_chunks = (int)total;
    }
    fill_chunks(pre, offs, S, n_vis, chunk, small, capacity, chunks, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kScanThreads)
chunk_prefix(const int64_t *__restrict__ offs, int S, int64_t n_vis, int chunk, int small,
             int *__restrict__ prefix, int *__restrict__ n_chunks, int capacity,
             int *__restrict__ work_counter, DeviceStatus *__restrict__ status)
{
    pdl_trigger();                          // the chunk table kernel may be scheduled now
    const long long total = scan_chunks(offs, S, n_vis, chunk, small, prefix, capacity, true, status);
    if (threadIdx.x == 0) {
        *work_counter = 0;
        *n_chunks = (int)total;
    }
}

__global__ void chunk_fill(const int *__restrict__ prefix, const int64_t *__restrict__ offs,
                           int S, int64_t n_vis, int chunk, int small, int capacity,
                           ChunkDesc *__restrict__ chunks)
{
    pdl_trigger();
    pdl_wait();                             // prefix[] complete
    fill_chunks(prefix, offs, S, n_vis, chunk, small, capacity, chunks, blockIdx.x, gridDim.x);
}

}  // namespace

cudaError_t launch_schedule(cudaStream_t st, const int64_t *vis_offsets, int n_subgrids,
                            int64_t n_vis, int chunk, int small, int *prefix, int *n_chunks,
                            ChunkDesc *chunks, int capacity, int *work_counter,
                            DeviceStatus *status)
{
    if (n_subgrids <= kSchedMaxS) {
        const int blocks = n_subgrids < 1 ? 1 : (n_subgrids < kSchedMaxBlocks ? n_subgrids : kSchedMaxBlocks);
        chunk_schedule<<<blocks, kSchedThreads, 0, st>>>(vis_offsets, n_subgrids, n_vis, chunk, small, n_chunks,
                                                        capacity, work_counter, status, chunks);
        return cudaGetLastError();
    }
    chunk_prefix<<<1, kScanThreads, 0, st>>>(vis_offsets, n_subgrids, n_vis, chunk, small, prefix, n_chunks,
                                             capacity, work_counter, status);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess)
        return err;
    const int blocks = n_subgrids < 4096 ? n_subgrids : 4096;
    return launch_pdl(chunk_fill, dim3(blocks), dim3(256), 0, st, (const int *)prefix, vis_offsets,
                      n_subgrids, n_vis, chunk, small, capacity, chunks);
}

}  // namespace dg
