// Adjoint of degridding (gridding): scatter every visibility back onto its
// 8 x 8 x 4 footprint with the weights of the forward sum,
//   sub[s][y0+b][x0+a][z0+c] += g_v[b] g_u[a] g_w[c] * vis[i].
// The weights are real, so this is the exact transpose of degrid.cu.
//
// Same work decomposition as the forward kernel: a warp walks a chunk of one
// subgrid in batches of 32 visibilities, lane i staging the coordinates, GCF
// rows and value of visibility i in shared memory.  Lane (a, c) then keeps
// an 8-row accumulator A[b] for the current footprint in registers and adds
// each visibility's contribution with packed FP32 FMAs.  Only when the
// footprint start changes (or the chunk ends) does the warp flush A to global
// memory with vector float2 atomics: 8 coalesced 256-byte atomic rows per
// footprint, instead of 256 atomics per visibility.  On a dense list
// hundreds of consecutive visibilities share a footprint, so atomic traffic
// is a small fraction of the FMA work.
#include "internal.cuh"

namespace dg {
namespace {

constexpr int kMaxWarps = 8;

struct alignas(16) WarpTile {
    float4 gv[kWarp][2];
    float gu[kWarp][kUV];
    float gw[kWarp][kW];
    float2 y[kWarp];
    int key[kWarp];
};

__device__ __forceinline__ float2 bcast2(float x) { return make_float2(x, x); }

__device__ __forceinline__ void flush(float2 (&A)[kUV], float2 *dst, int row_stride)
{
#pragma unroll
    for (int b = 0; b < kUV; ++b) {
        atomicAdd(dst + (int64_t)b * row_stride, A[b]);
        A[b] = make_float2(0.f, 0.f);
    }
}

__global__ void __launch_bounds__(kMaxWarps * kWarp)
adjoint_kernel(const Geometry g, const double *__restrict__ uvw,
               const float2 *__restrict__ vis_in, const float4 *__restrict__ guv4,
               const float4 *__restrict__ gw4, const Schedule sched,
               float2 *__restrict__ sub_out, DeviceStatus *__restrict__ status)
{
    extern __shared__ WarpTile tiles[];
    const int lane = threadIdx.x & 31;
    WarpTile &t = tiles[threadIdx.x >> 5];
    const int a = lane >> 2, c = lane & 3;
    const int lane_off = a * g.nz + c;
    const int total = *sched.n_chunks;

    for (;;) {
        int k = 0;
        if (lane == 0)
            k = atomicAdd(sched.work_counter, 1);
        k = __shfl_sync(kFull, k, 0);
        if (k >= total)
            break;
        const ChunkDesc cd = sched.chunks[k];
        const int64_t lo = cd.lo;
        const int64_t hi = lo + cd.n;
        float2 *const sub = sub_out + (int64_t)cd.s * g.plane + lane_off;

        int cur = -1;           // footprint key accumulated in A (-1: none)
        float2 A[kUV];
#pragma unroll
        for (int b = 0; b < kUV; ++b)
            A[b] = make_float2(0.f, 0.f);

        for (int64_t b0 = lo; b0 < hi; b0 += kWarp) {
            const int64_t idx = b0 + lane;
            const bool in = idx < hi;
            VisCoords vc;
            bool valid = false;
            float2 y = make_float2(0.f, 0.f);
            if (in) {
                const double u = __ldg(uvw + 3 * idx);
                const double v = __ldg(uvw + 3 * idx + 1);
                const double w = __ldg(uvw + 3 * idx + 2);
                valid = visibility_coords(u, v, w, g, vc);
                y = __ldg(vis_in + idx);
            }
            const int key = valid ? (vc.y0 * g.nx + vc.x0) * g.nz + vc.z0 : -1;
            const int fu = valid ? vc.fu : 0, fv = valid ? vc.fv : 0, fw = valid ? vc.fw : 0;
            t.gv[lane][0] = __ldg(guv4 + 2 * fv);
            t.gv[lane][1] = __ldg(guv4 + 2 * fv + 1);
            reinterpret_cast<float4 *>(t.gu[lane])[0] = __ldg(guv4 + 2 * fu);
            reinterpret_cast<float4 *>(t.gu[lane])[1] = __ldg(guv4 + 2 * fu + 1);
            reinterpret_cast<float4 *>(t.gw[lane])[0] = __ldg(gw4 + fw);
            t.y[lane] = y;
            t.key[lane] = key;
            const unsigned bad = __ballot_sync(kFull, in && !valid);
            if (lane == 0 && bad)
                atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
            __syncwarp();

            const int nv = (int)min((int64_t)kWarp, hi - b0);
            for (int v = 0; v < nv; ++v) {
                const int kv = t.key[v];
                if (kv != cur) {                    // warp-uniform
                    if (cur >= 0)
                        flush(A, sub + cur, g.row_stride);
                    cur = kv;
                }
                if (kv < 0)
                    continue;
                const float4 ga = t.gv[v][0], gb = t.gv[v][1];
                const float wac = t.gu[v][a] * t.gw[v][c];
                const float2 yw = __fmul2_rn(t.y[v], bcast2(wac));
                A[0] = __ffma2_rn(yw, bcast2(ga.x), A[0]);
                A[1] = __ffma2_rn(yw, bcast2(ga.y), A[1]);
                A[2] = __ffma2_rn(yw, bcast2(ga.z), A[2]);
                A[3] = __ffma2_rn(yw, bcast2(ga.w), A[3]);
                A[4] = __ffma2_rn(yw, bcast2(gb.x), A[4]);
                A[5] = __ffma2_rn(yw, bcast2(gb.y), A[5]);
                A[6] = __ffma2_rn(yw, bcast2(gb.z), A[6]);
                A[7] = __ffma2_rn(yw, bcast2(gb.w), A[7]);
            }
            __syncwarp();
        }
        if (cur >= 0)
            flush(A, sub + cur, g.row_stride);
    }
}

}  // namespace
}  // namespace dg

cudaError_t dg_launch_adjoint(degrid_plan *p, cudaStream_t st, const double *uvw,
                              const int64_t *vis_offsets, const float *vis_in,
                              float *sub_out, int grid_blocks)
{
    using namespace dg;
    (void)vis_offsets;
    Schedule sched{p->chunks, p->n_chunks, p->work_counter};
    const int threads = p->warps_per_block * kWarp;
    const size_t smem = sizeof(WarpTile) * p->warps_per_block;
    adjoint_kernel<<<grid_blocks, threads, smem, st>>>(
        p->geo, uvw, reinterpret_cast<const float2 *>(vis_in),
        reinterpret_cast<const float4 *>(p->guv), reinterpret_cast<const float4 *>(p->gw),
        sched, reinterpret_cast<float2 *>(sub_out), p->status);
    return cudaGetLastError();
}

int dg_max_blocks_per_sm_adjoint(degrid_plan *p)
{
    using namespace dg;
    int n = 0;
    const size_t smem = sizeof(WarpTile) * p->warps_per_block;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_kernel,
                                                      p->warps_per_block * kWarp, smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}
