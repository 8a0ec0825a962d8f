// Work decomposition for the persistent kernels.
//
// The paper launches a grid of max_S(N_vis,S / N_b) x S thread blocks
// (Eq. 1) and notes that uneven visibility counts leave most of it idle.
// Here the visibilities of every subgrid are cut into chunks of `chunk`
// visibilities (a chunk never straddles two subgrids), the chunks of all
// subgrids are numbered consecutively, and a persistent grid claims them
// with an atomic counter, so the load is balanced whatever the counts are.
//
// The chunk table is built on the device, so no host synchronisation is
// needed and the whole call can be captured in a CUDA graph.  For up to
// kSchedMaxS subgrids one kernel does it: every block scans
// ceil(count_s / chunk) over all subgrids into its shared memory (the scan
// is small and every block gets the same result), block 0 also validates
// vis_offsets and resets the work counter, and each block writes the chunk
// descriptors (s, count, first visibility) of its share of the subgrids.
// Larger stacks take two kernels: chunk_prefix (one block scans into
// prefix[S + 1] in global memory) and chunk_fill (the descriptors).
#include "internal.cuh"

namespace dg {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kSchedMaxS = 4096;            // subgrids the one-kernel schedule scans in shared memory
constexpr int kSchedMaxBlocks = 1024;
constexpr int kSchedThreads = 256;          // the one-kernel schedule's blocks

// Exclusive scan of ceil(count_s / chunk) over s < S into pre[0..S] (shared
// or global memory), each entry clamped to `capacity`; every thread of the
// block gets the (clamped) total.  With `lead` the block records malformed
// offsets and an overflowing total in the status flags.
__device__ long long scan_chunks(const int64_t *__restrict__ offs, int S, int64_t n_vis, int chunk,
                                 int *pre, int capacity, bool lead, DeviceStatus *status)
{
    __shared__ long long warp_sums[kScanThreads / kWarp];
    __shared__ long long carry_sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        carry_sh = 0;
        if (lead && (offs[0] != 0 || offs[S] != n_vis))
            atomicOr(&status->flags, kFlagOffsets);
    }
    __syncthreads();
    const int nt = blockDim.x;              // a multiple of 32, at most kScanThreads
    for (int base = 0; base < S; base += nt) {
        const int s = base + tid;
        long long cnt = 0;
        if (s < S) {
            const int64_t lo = offs[s], hi = offs[s + 1];
            const bool ok = lo >= 0 && lo <= hi && hi <= n_vis;
            if (!ok) {
                if (lead)
                    atomicOr(&status->flags, kFlagOffsets);
            } else {
                cnt = (hi - lo + chunk - 1) / chunk;
            }
        }
        // inclusive scan: within warps, then over warp totals
        long long x = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(kFull, x, d);
            if (lane >= d)
                x += y;
        }
        if (lane == 31)
            warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long t = warp_sums[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long y = __shfl_up_sync(kFull, t, d);
                if (lane >= d)
                    t += y;
            }
            warp_sums[lane] = t;        // inclusive over warps
        }
        __syncthreads();
        const long long before = carry_sh + (wid ? warp_sums[wid - 1] : 0) + x - cnt;
        if (s < S)
            pre[s] = (int)min(before, (long long)capacity);
        __syncthreads();
        if (tid == 0)
            carry_sh += warp_sums[nt / kWarp - 1];
        __syncthreads();
    }
    long long total = carry_sh;
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

// Descriptors of the chunks of subgrids s = first, first + step, ...
__device__ __forceinline__ void fill_chunks(const int *pre, const int64_t *__restrict__ offs, int S, int chunk,
                                            ChunkDesc *__restrict__ chunks, int first, int step)
{
    for (int s = first; s < S; s += step) {
        const int lo = pre[s], hi = pre[s + 1];
        const int64_t vis_lo = offs[s], vis_hi = offs[s + 1];
        for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
            const int64_t first_vis = vis_lo + (int64_t)(k - lo) * chunk;
            const int64_t last = min(first_vis + (int64_t)chunk, vis_hi);
            chunks[k] = ChunkDesc{s, (int)(last - first_vis), (long long)first_vis};
        }
    }
}

__global__ void __launch_bounds__(kSchedThreads)
chunk_schedule(const int64_t *__restrict__ offs, int S, int64_t n_vis, int chunk, int *__restrict__ n_chunks,
               int capacity, int *__restrict__ work_counter, DeviceStatus *__restrict__ status,
               ChunkDesc *__restrict__ chunks)
{
    __shared__ int pre[kSchedMaxS + 1];
    pdl_trigger();                          // the summing kernel may be scheduled now
    const bool lead = blockIdx.x == 0;
    const long long total = scan_chunks(offs, S, n_vis, chunk, pre, capacity, lead, status);
    if (lead && threadIdx.x == 0) {
        *work_counter = 0;
        *n_chunks = (int)total;
    }
    fill_chunks(pre, offs, S, chunk, chunks, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kScanThreads)
chunk_prefix(const int64_t *__restrict__ offs, int S, int64_t n_vis, int chunk,
             int *__restrict__ prefix, int *__restrict__ n_chunks, int capacity,
             int *__restrict__ work_counter, DeviceStatus *__restrict__ status)
{
    pdl_trigger();                          // the chunk table kernel may be scheduled now
    const long long total = scan_chunks(offs, S, n_vis, chunk, prefix, capacity, true, status);
    if (threadIdx.x == 0) {
        *work_counter = 0;
        *n_chunks = (int)total;
    }
}

__global__ void chunk_fill(const int *__restrict__ prefix, const int64_t *__restrict__ offs,
                           int S, int chunk, ChunkDesc *__restrict__ chunks)
{
    pdl_trigger();
    pdl_wait();                             // prefix[] complete
    fill_chunks(prefix, offs, S, chunk, chunks, blockIdx.x, gridDim.x);
}

}  // namespace

cudaError_t launch_schedule(cudaStream_t st, const int64_t *vis_offsets, int n_subgrids,
                            int64_t n_vis, int chunk, int *prefix, int *n_chunks,
                            ChunkDesc *chunks, int capacity, int *work_counter,
                            DeviceStatus *status)
{
    if (n_subgrids <= kSchedMaxS) {
        const int blocks = n_subgrids < 1 ? 1 : (n_subgrids < kSchedMaxBlocks ? n_subgrids : kSchedMaxBlocks);
        chunk_schedule<<<blocks, kSchedThreads, 0, st>>>(vis_offsets, n_subgrids, n_vis, chunk, n_chunks,
                                                        capacity, work_counter, status, chunks);
        return cudaGetLastError();
    }
    chunk_prefix<<<1, kScanThreads, 0, st>>>(vis_offsets, n_subgrids, n_vis, chunk, prefix, n_chunks,
                                             capacity, work_counter, status);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess)
        return err;
    const int blocks = n_subgrids < 4096 ? n_subgrids : 4096;
    return launch_pdl(chunk_fill, dim3(blocks), dim3(256), 0, st, (const int *)prefix, vis_offsets,
                      n_subgrids, chunk, chunks);
}

}  // namespace dg
