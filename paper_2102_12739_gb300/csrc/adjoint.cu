// Adjoint of degridding (gridding): scatter every visibility back onto its
// 8 x 8 x 4 footprint with the weights of the forward sum,
//   sub[s][y0+b][x0+a][z0+c] += g_v[b] g_u[a] g_w[c] * vis[i].
// The weights are real, so this is the exact transpose of degrid.cu.
//
// The batch pipeline is the forward kernel's (pipeline.cuh), with the
// visibility values staged next to the coordinates and GCF rows.  The
// scatter is factored like the forward sum: for a run of visibilities that
// share the footprint start and the w-kernel row,
//   sub[y0+b][x0+a][z0+c] += g_w[c] T[b][a],   T[b][a] = sum_i g_v,i[b] g_u,i[a] y_i,
// so each visibility adds 72 complex x real products into registers and the
// subgrid is touched only when the run ends.  Each quarter-warp handles one
// visibility per step (4 per step, 8 steps per batch); lane q of a quarter
// keeps the column T[0..7][q] of its quarter's partial sum and, when the run
// ends, flushes it with 32 vector float2 atomics (sub += g_w[c] T[b][q] for
// c = 0..3, b = 0..7).  Dense lists have runs of hundreds of visibilities, so
// the atomics are a small fraction of the work; a batch whose 32 visibilities
// share one run takes a branch-free path.
#include "pipeline.cuh"

namespace dg {
namespace {

#ifndef DG_ADJOINT_MIN_BLOCKS
#define DG_ADJOINT_MIN_BLOCKS 3
#endif

constexpr int kMaxWarps = 8;

struct alignas(128) WarpSmem {
    Stage st[2];
};

// Column accumulation of one run, owned by one quarter-warp.
struct Run {
    float2 T[8];
    int key;    // footprint start, -1 when nothing is accumulated
    int fw;
};

__device__ __forceinline__ void run_reset(Run &R)
{
#pragma unroll
    for (int b = 0; b < 8; ++b)
        R.T[b] = make_float2(0.f, 0.f);
    R.key = -1;
}

// sub[y0 + b][x0 + q][z0 + c] += g_w[c] T[b][q] for the run's footprint.
__device__ __forceinline__ void run_flush(Run &R, float2 *__restrict__ sub_s, int q, const Geometry &g,
                                          const float4 *wtab, const float *__restrict__ gwt)
{
    if (R.key < 0)
        return;
    const float4 gw = wtab ? wtab[R.fw] : __ldg(reinterpret_cast<const float4 *>(gwt) + R.fw);
    float2 *col = sub_s + R.key + (int64_t)q * g.nz;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        float2 *e = col + (int64_t)b * g.row_stride;
        const float2 t = R.T[b];
        atomicAdd(e, make_float2(t.x * gw.x, t.y * gw.x));
        atomicAdd(e + 1, make_float2(t.x * gw.y, t.y * gw.y));
        atomicAdd(e + 2, make_float2(t.x * gw.z, t.y * gw.z));
        atomicAdd(e + 3, make_float2(t.x * gw.w, t.y * gw.w));
    }
    run_reset(R);
}

// T[b] += g_v,r[b] * (g_u,r[q] * y_r): 18 FP32 operations.
__device__ __forceinline__ void run_add(Run &R, const Stage &S, int r, int q)
{
    const float4 v0 = reinterpret_cast<const float4 *>(S.gv[r])[0];
    const float4 v1 = reinterpret_cast<const float4 *>(S.gv[r])[1];
    const float gu = S.gu[r][q];
    const float2 y = S.y[r];
    const float wr = y.x * gu, wi = y.y * gu;
    const float gv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        R.T[b].x = fmaf(gv[b], wr, R.T[b].x);
        R.T[b].y = fmaf(gv[b], wi, R.T[b].y);
    }
}

__global__ void __launch_bounds__(kMaxWarps * kWarp, DG_ADJOINT_MIN_BLOCKS)
adjoint_kernel(const Geometry g, const double *__restrict__ uvw, const float2 *__restrict__ vis_in,
               const float *__restrict__ guv, const float *__restrict__ gwt, const Schedule sched,
               float2 *__restrict__ sub_out, DeviceStatus *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(smem_raw + wtable_bytes(g))[threadIdx.x >> 5];
    const float4 *wtab = load_wtable(g, gwt, smem_raw);
    const int lane = threadIdx.x & 31;
    const int quarter = lane >> 3, q = lane & 7;

    Claimer claimer(sched, lane, Prefetch{uvw, 3 * (int)sizeof(double), vis_in, (int)sizeof(float2)});
    Batch bB = claimer.claim();
    if (bB.n == 0)
        return;
    issue_batch(bB, load_uvw(uvw, bB, lane), g, ws.st[0], guv, gwt, wtab, lane, status, vis_in);
    Batch bC = claimer.advance(bB);
    Coords3 cC = load_uvw(uvw, bC, lane);

    int stage = 0;
    Run R;
    run_reset(R);
    int run_s = -1;                     // subgrid of the run in R
    float2 *sub_s = sub_out;

    while (bB.n > 0) {
        const Batch bA = bB;
        const int sA = stage;
        bB = bC;
        if (bB.n > 0)
            issue_batch(bB, cC, g, ws.st[sA ^ 1], guv, gwt, wtab, lane, status, vis_in);
        bC = claimer.advance(bC);
        cC = load_uvw(uvw, bC, lane);
        if (bB.n > 0)
            cp_async_wait<1>();
        else
            cp_async_wait<0>();
        __syncwarp();

        const Stage &S = ws.st[sA];
        if (bA.s != run_s) {
            run_flush(R, sub_s, q, g, wtab, gwt);
            run_s = bA.s;
            sub_s = sub_out + (int64_t)bA.s * g.plane;
        }
        if (S.uniform) {
            const int k0 = S.key[0], f0 = S.fw[0];
            if (k0 != R.key || f0 != R.fw) {
                run_flush(R, sub_s, q, g, wtab, gwt);
                R.key = k0;
                R.fw = f0;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
                run_add(R, S, 4 * t + quarter, q);
        } else {
#pragma unroll 1
            for (int t = 0; t < 8; ++t) {
                const int r = 4 * t + quarter;
                const int kv = S.key[r], fv = S.fw[r];
                if (kv < 0)
                    continue;
                if (kv != R.key || fv != R.fw) {
                    run_flush(R, sub_s, q, g, wtab, gwt);
                    R.key = kv;
                    R.fw = fv;
                }
                run_add(R, S, r, q);
            }
        }
        __syncwarp();
        stage ^= 1;
    }
    run_flush(R, sub_s, q, g, wtab, gwt);
}

size_t smem_bytes(const degrid_plan *p)
{
    return wtable_bytes_host(p->geo) + sizeof(WarpSmem) * (size_t)p->warps_per_block;
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
    const size_t smem = smem_bytes(p);
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    adjoint_kernel<<<grid_blocks, p->warps_per_block * kWarp, smem, st>>>(
        p->geo, uvw, reinterpret_cast<const float2 *>(vis_in), p->guv, p->gw, sched,
        reinterpret_cast<float2 *>(sub_out), p->status);
    return cudaGetLastError();
}

int dg_max_blocks_per_sm_adjoint(degrid_plan *p)
{
    using namespace dg;
    int n = 0;
    const size_t smem = smem_bytes(p);
    if (cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, adjoint_kernel, p->warps_per_block * kWarp,
                                                      smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}
