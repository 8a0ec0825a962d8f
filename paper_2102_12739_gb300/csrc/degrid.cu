// Degridding kernel (paper Section "Implementation": kernel D1 and its
// variants), re-designed for sm_103a.
//
// Work decomposition (pipeline.cuh).  A persistent grid of warps walks chunks
// of consecutive visibilities of one subgrid in batches of 32.  Per batch
// three stages overlap across consecutive batches of a warp:
//  1. the FP64 coordinates of batch n + 2 are loaded into registers;
//  2. batch n + 1 is snapped and its GCF rows are copied into the warp's
//     shared-memory stage with cp.async;
//  3. batch n is summed from the stage that arrived.
//
// Footprint sum.  The separable weights let the 8 x 8 x 4 sum be taken in
// three contractions,
//     V = sum_b g_v[b] sum_a g_u[a] M[b][a],   M[b][a] = sum_c g_w[c] s[y0+b][x0+a][z0+c],
// and M depends only on the footprint start and the w-kernel row.  On a dense
// list hundreds of consecutive visibilities share both (the reuse the paper
// notes for D1), so M is computed once per run and each visibility then costs
// 72 complex x real products instead of 256.  Each quarter-warp computes one
// visibility (4 per step, 8 steps per batch); lane q of a quarter keeps the
// column M[0..7][q] in registers, accumulates along v (b) as D1 does, and
// scales by g_u[q].  A batch whose 32 visibilities share one footprint and
// one w row takes a branch-free path; otherwise each quarter checks, and
// rebuilds its M when its visibility needs another one (so every input is
// handled, at up to 82 products per visibility when nothing is shared).
// Scalar FP32 FMAs: packed FFMA2 with three distinct register pairs ran at
// about half the FP32 peak on this part.
//
// Reduction and output.  The 8 partials of a quarter are reduced with a
// transposing butterfly (3 shuffle levels that halve the live values), after
// which every lane holds one whole visibility; the warp writes its 32
// results into one contiguous 256-byte segment (the paper's bulk contiguous
// write-out, without the shared-memory staging).
#include "pipeline.cuh"

namespace dg {
namespace {

#ifndef DG_DEGRID_MIN_BLOCKS
#define DG_DEGRID_MIN_BLOCKS 3   // resident CTAs per SM the register budget is sized for
#endif

constexpr int kMaxWarps = 8;                // per CTA
struct alignas(128) WarpSmem {
    Stage st[2];
    float2 part[8][kWarp];      // per-step partials on the mixed path
};

// ---- the factored sum -------------------------------------------------------

// M[b] = sum_c g_w[c] s[y0 + b][x0 + q][z0 + c] for b = 0..7 (this lane's
// column q of the footprint with origin `key` in the subgrid at `base`).
template <int DT>
__device__ __forceinline__ void build_column(float2 (&M)[8], const void *sub, int64_t base, int key,
                                             int q, const float4 &gw, const Geometry &g)
{
    const int64_t col = base + key + (int64_t)q * g.nz;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int64_t e = col + (int64_t)b * g.row_stride;
        const float2 s0 = Storage<DT>::load(sub, e), s1 = Storage<DT>::load(sub, e + 1);
        const float2 s2 = Storage<DT>::load(sub, e + 2), s3 = Storage<DT>::load(sub, e + 3);
        M[b].x = fmaf(s3.x, gw.w, fmaf(s2.x, gw.z, fmaf(s1.x, gw.y, s0.x * gw.x)));
        M[b].y = fmaf(s3.y, gw.w, fmaf(s2.y, gw.z, fmaf(s1.y, gw.y, s0.y * gw.x)));
    }
}

// This lane's part of visibility r: g_u[q] * sum_b g_v[b] M[b] (18 FP32 ops).
__device__ __forceinline__ float2 apply_column(const float2 (&M)[8], const Stage &S, int r, int q)
{
    const float4 v0 = reinterpret_cast<const float4 *>(S.gv[r])[0];
    const float4 v1 = reinterpret_cast<const float4 *>(S.gv[r])[1];
    const float gu = S.gu[r][q];
    float re = M[0].x * v0.x, im = M[0].y * v0.x;
    re = fmaf(M[1].x, v0.y, re);
    im = fmaf(M[1].y, v0.y, im);
    re = fmaf(M[2].x, v0.z, re);
    im = fmaf(M[2].y, v0.z, im);
    re = fmaf(M[3].x, v0.w, re);
    im = fmaf(M[3].y, v0.w, im);
    re = fmaf(M[4].x, v1.x, re);
    im = fmaf(M[4].y, v1.x, im);
    re = fmaf(M[5].x, v1.y, re);
    im = fmaf(M[5].y, v1.y, im);
    re = fmaf(M[6].x, v1.z, re);
    im = fmaf(M[6].y, v1.z, im);
    re = fmaf(M[7].x, v1.w, re);
    im = fmaf(M[7].y, v1.w, im);
    return make_float2(re * gu, im * gu);
}

// Transposing butterfly over the 8 lanes of a quarter: on entry P[t] is this
// lane's partial of step t; on exit the lane returns the total of step q.
__device__ __forceinline__ float2 quarter_reduce(float2 (&P)[8], int q)
{
#pragma unroll
    for (int h = 4; h >= 1; h >>= 1) {
        const bool up = (q & h) != 0;
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
__global__ void __launch_bounds__(kMaxWarps * kWarp, DG_DEGRID_MIN_BLOCKS)
degrid_kernel(const Geometry g, const void *__restrict__ subgrids, const float *__restrict__ scale,
              const double *__restrict__ uvw, const float *__restrict__ guv,
              const float *__restrict__ gwt, const Schedule sched, float2 *__restrict__ vis_out,
              DeviceStatus *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // [w table (optional)] [one WarpSmem per warp]
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(smem_raw + wtable_bytes(g))[threadIdx.x >> 5];
    const float4 *wtab = load_wtable(g, gwt, smem_raw);
    const int lane = threadIdx.x & 31;
    const int quarter = lane >> 3, q = lane & 7;

    Claimer claimer(sched, lane);
    Batch bB = claimer.claim();         // rows in flight
    if (bB.n == 0)
        return;
    issue_batch(bB, load_uvw(uvw, bB, lane), g, ws.st[0], guv, gwt, wtab, lane, status);
    Batch bC = claimer.advance(bB);     // coordinates in registers
    Coords3 cC = load_uvw(uvw, bC, lane);

    int stage = 0;
    float2 M[8];                        // footprint column M[0..7][q] of (m_key, m_fw, m_s)
    int m_key = -2, m_fw = -1, m_s = -1;
#pragma unroll
    for (int b = 0; b < 8; ++b)
        M[b] = make_float2(0.f, 0.f);

    while (bB.n > 0) {
        const Batch bA = bB;            // summed in this iteration
        const int sA = stage;
        bB = bC;
        if (bB.n > 0)
            issue_batch(bB, cC, g, ws.st[sA ^ 1], guv, gwt, wtab, lane, status);
        bC = claimer.advance(bC);
        cC = load_uvw(uvw, bC, lane);
        if (bB.n > 0)
            cp_async_wait<1>();         // the stage of batch A; batch B may stay in flight
        else
            cp_async_wait<0>();
        __syncwarp();

        const Stage &S = ws.st[sA];
        if (bA.s != m_s) {
            m_s = bA.s;
            m_key = -2;
        }
        const int64_t base = (int64_t)bA.s * g.plane;
        float2 P[8];
        if (S.uniform) {
            const int k0 = S.key[0], f0 = S.fw[0];
            if (k0 != m_key || f0 != m_fw) {
                build_column<DT>(M, subgrids, base, k0, q, reinterpret_cast<const float4 *>(S.gw)[0], g);
                m_key = k0;
                m_fw = f0;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
                P[t] = apply_column(M, S, 4 * t + quarter, q);
        } else {
#pragma unroll 1
            for (int t = 0; t < 8; ++t) {
                const int r = 4 * t + quarter;
                const int kv = S.key[r], fv = S.fw[r];
                if (kv >= 0 && (kv != m_key || fv != m_fw)) {
                    build_column<DT>(M, subgrids, base, kv, q, reinterpret_cast<const float4 *>(S.gw)[r], g);
                    m_key = kv;
                    m_fw = fv;
                }
                ws.part[t][lane] = kv >= 0 ? apply_column(M, S, r, q) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
                P[t] = ws.part[t][lane];
        }
        float2 V = quarter_reduce(P, q);
        const int r_out = 4 * q + quarter;
        if (DT != DG_C64) {
            const float sc = __ldg(scale + bA.s);
            V = __fmul2_rn(V, make_float2(sc, sc));
        }
        if (r_out < bA.n)
            vis_out[bA.b0 + r_out] = V;
        __syncwarp();
        stage ^= 1;
    }
}

size_t smem_bytes(const degrid_plan *p, int warps)
{
    return wtable_bytes_host(p->geo) + sizeof(WarpSmem) * (size_t)warps;
}

template <int DT>
cudaError_t launch(degrid_plan *p, cudaStream_t st, const void *subgrids, const float *scale,
                   const double *uvw, float2 *out, const Schedule &sched, int grid_blocks)
{
    const int threads = p->warps_per_block * kWarp;
    const size_t smem = smem_bytes(p, p->warps_per_block);
    cudaError_t e = cudaFuncSetAttribute(degrid_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess)
        return e;
    degrid_kernel<DT><<<grid_blocks, threads, smem, st>>>(p->geo, subgrids, scale, uvw, p->guv,
                                                           p->gw, sched, out, p->status);
    return cudaGetLastError();
}

template <int DT>
int max_blocks(degrid_plan *p)
{
    int n = 0;
    const size_t smem = smem_bytes(p, p->warps_per_block);
    if (cudaFuncSetAttribute(degrid_kernel<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, degrid_kernel<DT>,
                                                      p->warps_per_block * kWarp, smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace
}  // namespace dg

cudaError_t dg_launch_degrid(degrid_plan *p, cudaStream_t st, const void *subgrids,
                             const float *scale, const double *uvw, const int64_t *vis_offsets,
                             float *out_f, int grid_blocks)
{
    using namespace dg;
    (void)vis_offsets;
    Schedule sched{p->chunks, p->n_chunks, p->work_counter};
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

int dg_max_warps_per_block() { return dg::kMaxWarps; }
