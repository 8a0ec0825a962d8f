// Degridding kernel (paper Section "Implementation": kernel D1 and its
// variants), re-designed for sm_103a.
//
// Work decomposition.  A persistent grid of warps claims chunks of
// consecutive visibilities of one subgrid (schedule.cu, claims pipelined one
// chunk ahead) and walks each chunk in batches of 32 visibilities.  Per batch
// three stages overlap across consecutive batches of a warp:
//  1. the FP64 coordinates of batch n + 2 are loaded into registers;
//  2. for batch n + 1, lane i snaps visibility i (exact integer rint of the
//     coordinates, internal.cuh), records its footprint key and w-kernel row
//     and copies its g_u and g_v rows into the warp's shared-memory stage with
//     cp.async (the small w table lives in shared memory).  The paper's D1
//     likewise computes all coordinates of its N_b visibilities cooperatively
//     into shared memory before the sums;
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
#include "internal.cuh"

namespace dg {
namespace {

#ifndef DG_DEGRID_MIN_BLOCKS
#define DG_DEGRID_MIN_BLOCKS 3   // resident CTAs per SM the register budget is sized for
#endif

constexpr int kMaxWarps = 8;                // per CTA
constexpr int kBatch = 32;                  // visibilities per batch
constexpr int kUVRow = 8;                   // floats per uv table row (32 B)
constexpr int kWRow = 4;                    // floats per w table row (16 B)

struct alignas(128) Stage {
    float gu[kBatch][kUVRow];   // g_uv[fu], per visibility
    float gv[kBatch][kUVRow];   // g_uv[fv]
    float gw[kBatch][kWRow];    // g_w[fw]
    int key[kBatch];            // footprint start (y0 * nx + x0) * nz + z0, -1 invalid
    int fw[kBatch];             // w-kernel row
    int uniform;                // all 32 share one valid footprint and one w row
};

struct alignas(128) WarpSmem {
    Stage st[2];
    float2 part[8][kWarp];      // per-step partials on the mixed path
};

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

// ---- batch stream -----------------------------------------------------------

struct Batch {
    int s;          // subgrid
    int n;          // visibilities in this batch (1..32), 0 = none
    long long b0;   // first visibility
    long long end;  // end of the chunk
};

// Claims chunks with an atomic counter, one claim ahead: while a warp works
// on a chunk it already holds the descriptor of the next one, and the atomic
// for the one after that is in flight.
struct Claimer {
    const Schedule &sched;
    int total;
    int lane;
    int pend;           // lane 0: atomic result not yet consumed
    ChunkDesc next;     // descriptor of the chunk after the current one
    int next_valid;

    __device__ Claimer(const Schedule &sc, int lane_) : sched(sc), lane(lane_)
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
        if (lane == 0)
            pend = atomicAdd(sched.work_counter, 1);
        bt.s = cur.s;
        bt.b0 = cur.lo;
        bt.end = cur.lo + cur.n;
        bt.n = (int)min((long long)kBatch, bt.end - bt.b0);
        return bt;
    }

    __device__ Batch advance(const Batch &b)
    {
        if (b.n == 0)
            return b;
        Batch nb = b;
        nb.b0 = b.b0 + kBatch;
        if (nb.b0 >= b.end)
            return claim();
        nb.n = (int)min((long long)kBatch, b.end - nb.b0);
        return nb;
    }
};

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

// Stage 2 of a batch: coordinates, keys, w rows and the copies of the g_u /
// g_v rows (2 lanes per 32-byte row).
__device__ __forceinline__ void issue_batch(const Batch &b, const Coords3 &c, const Geometry &g,
                                            Stage &S, const float *__restrict__ guv,
                                            const float *__restrict__ gwt, const float4 *wtab,
                                            int lane, DeviceStatus *status)
{
    const bool in = lane < b.n;
    VisCoords vc;
    const bool valid = in && visibility_coords(c.u, c.v, c.w, g, vc);
    const int key = valid ? (vc.y0 * g.nx + vc.x0) * g.nz + vc.z0 : -1;
    const int fu = valid ? vc.fu : 0, fv = valid ? vc.fv : 0, fw = valid ? vc.fw : 0;
    S.key[lane] = key;
    S.fw[lane] = fw;
    const int key0 = __shfl_sync(kFull, key, 0), fw0 = __shfl_sync(kFull, fw, 0);
    const bool uniform = __all_sync(kFull, key == key0 && fw == fw0) && key0 >= 0;
    if (lane == 0)
        S.uniform = uniform;
    const unsigned bad = __ballot_sync(kFull, in && !valid);
    if (lane == 0 && bad)
        atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
    if (wtab)
        reinterpret_cast<float4 *>(S.gw)[lane] = wtab[fw];
    else
        cp_async16(smem_u32(S.gw[lane]), gwt + (size_t)fw * kWRow);
    const int half = lane & 1;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int r = (lane >> 1) + 16 * m;
        const int xu = __shfl_sync(kFull, fu, r);
        const int xv = __shfl_sync(kFull, fv, r);
        cp_async16(smem_u32(&S.gu[r][4 * half]), guv + (size_t)xu * kUVRow + 4 * half);
        cp_async16(smem_u32(&S.gv[r][4 * half]), guv + (size_t)xv * kUVRow + 4 * half);
    }
    cp_async_commit();
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
    const int wtab_bytes = g.w_table_rows > 0 ? ((g.w_table_rows * kWRow * 4 + 127) & ~127) : 0;
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(smem_raw + wtab_bytes)[threadIdx.x >> 5];
    const float4 *wtab = nullptr;
    if (wtab_bytes) {
        float4 *t = reinterpret_cast<float4 *>(smem_raw);
        const float4 *src = reinterpret_cast<const float4 *>(gwt);
        for (int i = threadIdx.x; i < g.w_table_rows; i += blockDim.x)
            t[i] = __ldg(src + i);
        __syncthreads();
        wtab = t;
    }
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
    const size_t wt = p->geo.w_table_rows > 0
                          ? ((size_t)p->geo.w_table_rows * kWRow * 4 + 127) & ~(size_t)127
                          : 0;
    return wt + sizeof(WarpSmem) * (size_t)warps;
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
