// Work decomposition for the persistent kernels.
//
// The paper launches a grid of max_S(N_vis,S / N_b) x S thread blocks
// (Eq. 1) and notes that uneven visibility counts leave most of it idle.
// Here the visibilities of every subgrid are cut into chunks of `chunk`
// visibilities (a chunk never straddles two subgrids), the chunks of all
// subgrids are numbered consecutively, and a persistent grid claims them
// with an atomic counter, so the load is balanced whatever the counts are.
//
// Two small kernels build the chunk table on the device, so no host
// synchronisation is needed and the whole call can be captured in a CUDA
// graph:
//   1. chunk_prefix: one block validates vis_offsets and scans
//      ceil(count_s / chunk) into prefix[S + 1];
//   2. chunk_fill: writes (s, count, first visibility) for every chunk.
// For small calls (few subgrids and chunks, bounded on the host) the block of
// chunk_prefix also writes the chunks, saving a launch.
#include "internal.cuh"

namespace dg {
namespace {

constexpr int kScanThreads = 1024;

constexpr int kSmallSubgrids = 32;          // one-launch schedule: at most this many subgrids
constexpr int kSmallChunks = 8192;          // and at most this many chunks (host bound)

__global__ void __launch_bounds__(kScanThreads)
chunk_prefix(const int64_t *__restrict__ offs, int S, int64_t n_vis, int chunk,
             int *__restrict__ prefix, int *__restrict__ n_chunks, int capacity,
             int *__restrict__ work_counter, DeviceStatus *__restrict__ status,
             ChunkDesc *__restrict__ fill_chunks)
{
    __shared__ long long warp_sums[kScanThreads / kWarp];
    __shared__ long long carry_sh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    pdl_trigger();                          // the chunk table (or sums) kernel may be scheduled now
    if (tid == 0) {
        carry_sh = 0;
        *work_counter = 0;
        if (S >= 0 && (offs[0] != 0 || offs[S] != n_vis))
            atomicOr(&status->flags, kFlagOffsets);
    }
    __syncthreads();
    for (int base = 0; base < S; base += kScanThreads) {
        const int s = base + tid;
        long long cnt = 0;
        if (s < S) {
            const int64_t lo = offs[s], hi = offs[s + 1];
            const bool ok = lo >= 0 && lo <= hi && hi <= n_vis;
            if (!ok)
                atomicOr(&status->flags, kFlagOffsets);
            else
                cnt = (hi - lo + chunk - 1) / chunk;
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
            prefix[s] = (int)min(before, (long long)capacity);
        __syncthreads();
        if (tid == 0)
            carry_sh += warp_sums[kScanThreads / kWarp - 1];
        __syncthreads();
    }
    if (tid == 0) {
        long long total = carry_sh;
        if (total > capacity) {
            atomicOr(&status->flags, kFlagCapacity);
            total = capacity;
        }
        prefix[S > 0 ? S : 0] = (int)total;
        *n_chunks = (int)total;
    }
    if (!fill_chunks)
        return;
    __syncthreads();                        // prefix[] visible to the whole block
    for (int s = 0; s < S; ++s) {
        const int lo = prefix[s], hi = prefix[s + 1];
        const int64_t vis_lo = offs[s], vis_hi = offs[s + 1];
        for (int k = lo + tid; k < hi; k += kScanThreads) {
            const int64_t first = vis_lo + (int64_t)(k - lo) * chunk;
            const int64_t last = min(first + (int64_t)chunk, vis_hi);
            fill_chunks[k] = ChunkDesc{s, (int)(last - first), (long long)first};
        }
    }
}

__global__ void chunk_fill(const int *__restrict__ prefix, const int64_t *__restrict__ offs,
                           int S, int chunk, ChunkDesc *__restrict__ chunks)
{
    pdl_trigger();
    pdl_wait();                             // prefix[] complete
    for (int s = blockIdx.x; s < S; s += gridDim.x) {
        const int lo = prefix[s], hi = prefix[s + 1];
        const int64_t vis_lo = offs[s], vis_hi = offs[s + 1];
        for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
            const int64_t first = vis_lo + (int64_t)(k - lo) * chunk;
            const int64_t last = min(first + (int64_t)chunk, vis_hi);
            chunks[k] = ChunkDesc{s, (int)(last - first), (long long)first};
        }
    }
}

}  // namespace

cudaError_t launch_schedule(cudaStream_t st, const int64_t *vis_offsets, int n_subgrids,
                            int64_t n_vis, int chunk, int *prefix, int *n_chunks,
                            ChunkDesc *chunks, int capacity, int *work_counter,
                            DeviceStatus *status)
{
    const bool small = n_subgrids <= kSmallSubgrids && n_vis / chunk + n_subgrids <= kSmallChunks;
    chunk_prefix<<<1, kScanThreads, 0, st>>>(vis_offsets, n_subgrids, n_vis, chunk, prefix,
                                             n_chunks, capacity, work_counter, status,
                                             small ? chunks : nullptr);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || n_subgrids == 0 || small)
        return err;
    const int blocks = n_subgrids < 4096 ? n_subgrids : 4096;
    return launch_pdl(chunk_fill, dim3(blocks), dim3(256), 0, st, (const int *)prefix, vis_offsets,
                      n_subgrids, chunk, chunks);
}

}  // namespace dg
