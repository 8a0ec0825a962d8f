// Degridding kernel (paper Section "Implementation", kernel D1 and its
// variants, re-designed for sm_103a).
//
// Work unit: one warp takes a chunk of consecutive visibilities of one
// subgrid (see schedule.cu) and walks it in batches of 32.
//
//  1. Coordinates.  Lane i snaps visibility i of the batch (exact integer
//     rint of the FP64 coordinates, internal.cuh) and stages its footprint
//     key and its three GCF rows (g_v[8], g_u[8], g_w[4], FP32) in the warp's
//     shared-memory tile.  The paper's D1 likewise computes all coordinates
//     of its N_b visibilities cooperatively into shared memory first.
//  2. Footprint sum.  The warp then visits the 32 visibilities in order.
//     Lane (a, c) = (lane / 4, lane % 4) keeps the 8 samples
//     s[y0 + b][x0 + a][z0 + c], b = 0..7, in registers and reloads them only
//     when the footprint start changes: consecutive visibilities of a dense
//     list share the footprint (the data reuse the paper notes for D1), so
//     the subgrid is read from L2 once per footprint, not once per
//     visibility.  Each lane accumulates along v (b), like D1, with packed
//     FP32 FMAs (one FFMA2 per complex x real product), then scales by
//     g_u[a] g_w[c].
//  3. Reduction.  The 32 lanes x 32 visibilities of partial sums are reduced
//     with a transposing butterfly (5 shuffle levels that halve the live
//     values), after which lane i holds visibility i: 2 shuffles per
//     visibility per lane instead of 10 for one warp reduction each.
//  4. Output.  Lane i writes visibility i, so the warp stores 256 contiguous
//     bytes (the paper's bulk contiguous write-out, without the staging).
#include "internal.cuh"

namespace dg {
namespace {

constexpr int kMaxWarps = 8;    // per CTA

struct alignas(16) WarpTile {
    float4 gv[kWarp][2];    // g_uv[fv][0..7]
    float gu[kWarp][kUV];   // g_uv[fu][0..7]
    float gw[kWarp][kW];    // g_w[fw][0..3]
    int key[kWarp];         // (y0 * nx + x0) * nz + z0, or -1 if invalid
};

__device__ __forceinline__ float2 bcast2(float x) { return make_float2(x, x); }

// Transposing butterfly: on entry lane l holds partials P[v] of visibility v
// (v = 0..31); on exit it returns sum over lanes of P[l].
__device__ __forceinline__ float2 transpose_reduce(float2 (&P)[kWarp], int lane)
{
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            float2 send = up ? P[j] : P[j + h];
            const float2 keep = up ? P[j + h] : P[j];
            send.x = __shfl_xor_sync(kFull, send.x, h);
            send.y = __shfl_xor_sync(kFull, send.y, h);
            P[j] = __fadd2_rn(keep, send);
        }
    }
    return P[0];
}

template <int DT>
__global__ void __launch_bounds__(kMaxWarps * kWarp)
degrid_kernel(const Geometry g, const void *__restrict__ subgrids,
              const float *__restrict__ scale, const double *__restrict__ uvw,
              const float4 *__restrict__ guv4, const float4 *__restrict__ gw4,
              const Schedule sched, float2 *__restrict__ vis_out,
              DeviceStatus *__restrict__ status)
{
    extern __shared__ WarpTile tiles[];
    const int lane = threadIdx.x & 31;
    WarpTile &t = tiles[threadIdx.x >> 5];
    const int a = lane >> 2, c = lane & 3;
    const int lane_off = a * g.nz + c;
    const int total = *sched.n_chunks;
    const int64_t *offs = sched.vis_offsets;

    for (;;) {
        int k = 0;
        if (lane == 0)
            k = atomicAdd(sched.work_counter, 1);
        k = __shfl_sync(kFull, k, 0);
        if (k >= total)
            break;
        const ChunkRef ref = sched.chunks[k];
        const int64_t lo = offs[ref.s] + (int64_t)ref.j * sched.chunk;
        const int64_t hi = min(lo + (int64_t)sched.chunk, offs[ref.s + 1]);
        const int64_t sub_base = (int64_t)ref.s * g.plane + lane_off;
        const float sc = (DT == DG_C64) ? 1.0f : __ldg(scale + ref.s);

        int cur = -2;               // footprint key held in B
        float2 B[kUV];
#pragma unroll
        for (int b = 0; b < kUV; ++b)
            B[b] = make_float2(0.f, 0.f);

        for (int64_t b0 = lo; b0 < hi; b0 += kWarp) {
            // ---- 1. coordinates and GCF rows of the batch -----------------
            const int64_t idx = b0 + lane;
            const bool in = idx < hi;
            VisCoords vc;
            bool valid = false;
            if (in) {
                const double u = __ldg(uvw + 3 * idx);
                const double v = __ldg(uvw + 3 * idx + 1);
                const double w = __ldg(uvw + 3 * idx + 2);
                valid = visibility_coords(u, v, w, g, vc);
            }
            const int key = valid ? (vc.y0 * g.nx + vc.x0) * g.nz + vc.z0 : -1;
            const int fu = valid ? vc.fu : 0, fv = valid ? vc.fv : 0, fw = valid ? vc.fw : 0;
            const float4 gu0 = __ldg(guv4 + 2 * fu), gu1 = __ldg(guv4 + 2 * fu + 1);
            const float4 gv0 = __ldg(guv4 + 2 * fv), gv1 = __ldg(guv4 + 2 * fv + 1);
            const float4 gwr = __ldg(gw4 + fw);
            t.gv[lane][0] = gv0;
            t.gv[lane][1] = gv1;
            reinterpret_cast<float4 *>(t.gu[lane])[0] = gu0;
            reinterpret_cast<float4 *>(t.gu[lane])[1] = gu1;
            reinterpret_cast<float4 *>(t.gw[lane])[0] = gwr;
            t.key[lane] = key;
            const unsigned bad = __ballot_sync(kFull, in && !valid);
            if (lane == 0 && bad)
                atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
            __syncwarp();

            // ---- 2. footprint sums -----------------------------------------
            float2 P[kWarp];
#pragma unroll
            for (int v = 0; v < kWarp; ++v) {
                const int kv = t.key[v];
                if (kv != cur) {                // warp-uniform
                    cur = kv;
                    if (kv >= 0) {
#pragma unroll
                        for (int b = 0; b < kUV; ++b)
                            B[b] = Storage<DT>::load(subgrids, sub_base + kv + (int64_t)b * g.row_stride);
                    } else {
#pragma unroll
                        for (int b = 0; b < kUV; ++b)
                            B[b] = make_float2(0.f, 0.f);
                    }
                }
                const float4 ga = t.gv[v][0], gb = t.gv[v][1];
                const float wac = t.gu[v][a] * t.gw[v][c];
                float2 acc = __fmul2_rn(B[0], bcast2(ga.x));
                acc = __ffma2_rn(B[1], bcast2(ga.y), acc);
                acc = __ffma2_rn(B[2], bcast2(ga.z), acc);
                acc = __ffma2_rn(B[3], bcast2(ga.w), acc);
                acc = __ffma2_rn(B[4], bcast2(gb.x), acc);
                acc = __ffma2_rn(B[5], bcast2(gb.y), acc);
                acc = __ffma2_rn(B[6], bcast2(gb.z), acc);
                acc = __ffma2_rn(B[7], bcast2(gb.w), acc);
                P[v] = __fmul2_rn(acc, bcast2(wac));
            }
            __syncwarp();

            // ---- 3./4. reduction and contiguous write-out ------------------
            float2 V = transpose_reduce(P, lane);
            if (DT != DG_C64)
                V = __fmul2_rn(V, bcast2(sc));
            if (in)
                vis_out[idx] = V;
        }
    }
}

template <int DT>
cudaError_t launch(degrid_plan *p, cudaStream_t st, const void *subgrids, const float *scale,
                   const double *uvw, float2 *out, const Schedule &sched, int grid_blocks)
{
    const int threads = p->warps_per_block * kWarp;
    const size_t smem = sizeof(WarpTile) * p->warps_per_block;
    degrid_kernel<DT><<<grid_blocks, threads, smem, st>>>(
        p->geo, subgrids, scale, uvw, reinterpret_cast<const float4 *>(p->guv),
        reinterpret_cast<const float4 *>(p->gw), sched, out, p->status);
    return cudaGetLastError();
}

template <int DT>
int max_blocks(degrid_plan *p)
{
    int n = 0;
    const size_t smem = sizeof(WarpTile) * p->warps_per_block;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, degrid_kernel<DT>,
                                                      p->warps_per_block * kWarp, smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace
}  // namespace dg

cudaError_t dg_launch_degrid(degrid_plan *p, cudaStream_t st, const void *subgrids,
                             const float *scale, const double *uvw,
                             const int64_t *vis_offsets, float *out_f, int grid_blocks)
{
    using namespace dg;
    Schedule sched{vis_offsets, p->chunks, p->n_chunks, p->work_counter, p->chunk};
    float2 *out = reinterpret_cast<float2 *>(out_f);
    switch (p->dtype) {
    case DG_C64:
        return launch<DG_C64>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    case DG_C32_F16:
        return launch<DG_C32_F16>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    case DG_C32_BF16:
        return launch<DG_C32_BF16>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    }
    return cudaErrorInvalidValue;
}

int dg_max_blocks_per_sm_degrid(degrid_plan *p)
{
    using namespace dg;
    switch (p->dtype) {
    case DG_C64: return max_blocks<DG_C64>(p);
    case DG_C32_F16: return max_blocks<DG_C32_F16>(p);
    case DG_C32_BF16: return max_blocks<DG_C32_BF16>(p);
    }
    return 1;
}
