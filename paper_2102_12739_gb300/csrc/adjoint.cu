// Adjoint of degridding (gridding): scatter every visibility back onto its
// 8 x 8 x 4 footprint with the weights of the forward sum,
//   sub[s][y0+b][x0+a][z0+c] += g_v[b] g_u[a] g_w[c] * vis[i]
// (or G[fv][fu][b][a] g_w[c] * vis[i] with a non-separable 2D G_uv table).
// The weights are real, so this is the exact transpose of degrid.cu.
//
// The pipeline is the forward kernel's (pipeline.cuh): steps of 64
// visibilities in two halves of 32; lane i of a half snaps visibility i,
// copies its g_u / g_v rows into the warp's stage and loads its value y_i a
// step ahead.  The scatter is factored like the
// forward sum: for a run of visibilities that share the footprint start and
// the w-kernel row,
//   sub[y0+b][x0+a][z0+c] += g_w[c] T[b][a],   T[b][a] = sum_i g_v,i[b] g_u,i[a] y_i,
// so each visibility adds 64 complex x real products into registers and the
// subgrid is touched only when the run ends.  Four lanes share a visibility:
// lane 8j + p keeps the rows T[2j][0..7], T[2j+1][0..7] (32 registers) of the
// visibilities 8k + p (pass k = 0..3) it handles.  At the end of a run the 8
// lanes p of each row pair add their partial T through shared memory (a
// transpose with XOR-swizzled 16-byte slots, free of bank conflicts) and lane
// 8j + p adds column a = p of rows 2j, 2j+1 to the subgrid with 8 float2
// atomics (c = 0..3).  Dense lists have runs of hundreds of visibilities, so
// the atomics are a small fraction of the work.  Halves whose 32
// visibilities share one run take a branch-free path.
#include "pipeline.cuh"

namespace dg {
namespace {

#ifndef DG_ADJOINT_MIN_BLOCKS
#define DG_ADJOINT_MIN_BLOCKS 2   // resident CTAs per SM the register budget (128) is sized for
#endif

constexpr int kMaxWarps = 8;

constexpr int kStepVis = 2 * kBatch;        // visibilities per pipeline step (two halves)

struct alignas(128) WarpSmem {
    RowStage st[2][2];          // [stage][half]
    float4 t[8][4][8];          // flush transpose: [p][j][slot a ^ p] = (T[2j][a], T[2j+1][a])
};

// Visibility value of this lane's visibility in batch b (0 past its end).
__device__ __forceinline__ float2 load_y(const float2 *__restrict__ vis, const Batch &b, int lane)
{
    return lane < b.n ? __ldg(vis + b.b0 + lane) : make_float2(0.f, 0.f);
}

// T[i][a] += g_u[a] * (g_v[2j + i] * y) for the visibility in row r.
__device__ __forceinline__ void accumulate(float2 (&T)[2][8], const RowStage &S, int r, int j, float2 y)
{
    const float4 u0 = S.u[r][row_half(r, 0)];
    const float4 u1 = S.u[r][row_half(r, 1)];
    const float2 v = reinterpret_cast<const float2 *>(&S.v[r][row_half(r, j >> 1)])[j & 1];
    const float gu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    const float2 w0 = __fmul2_rn(y, make_float2(v.x, v.x)), w1 = __fmul2_rn(y, make_float2(v.y, v.y));
    // packed (re, im) FMAs with a duplicated real weight (bitwise two scalar FMAs)
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        T[0][a] = __ffma2_rn(make_float2(gu[a], gu[a]), w0, T[0][a]);
        T[1][a] = __ffma2_rn(make_float2(gu[a], gu[a]), w1, T[1][a]);
    }
}

// 2D G_uv table: T[i][a] += G[blk][2j + i][a] * y for the visibility whose
// weight block is blk (16 weights of rows 2j, 2j + 1 read from the table).
__device__ __forceinline__ void accumulate_2d(float2 (&T)[2][8], const float *__restrict__ g2, int blk,
                                              int j, float2 y)
{
    const float4 *w = reinterpret_cast<const float4 *>(g2 + (size_t)blk * (kUV * kUV) + 2 * kUV * j);
    const float4 w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3);
    const float g0[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    const float g1[8] = {w2.x, w2.y, w2.z, w2.w, w3.x, w3.y, w3.z, w3.w};
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        T[0][a] = __ffma2_rn(make_float2(g0[a], g0[a]), y, T[0][a]);
        T[1][a] = __ffma2_rn(make_float2(g1[a], g1[a]), y, T[1][a]);
    }
}

// One visibility of a pass: the separable rows from the stage, or the 2D table.
template <bool T2D>
__device__ __forceinline__ void accumulate_vis(float2 (&T)[2][8], const RowStage &S,
                                               const float *__restrict__ g2, int r, int blk, int j,
                                               float2 y)
{
    if (T2D)
        accumulate_2d(T, g2, blk, j, y);
    else
        accumulate(T, S, r, j, y);
}

// Adds the run (key, fw) to the subgrid at sub_s and clears T.
__device__ __forceinline__ void flush(float2 (&T)[2][8], WarpSmem &ws, float2 *__restrict__ sub_s,
                                      int key, int fw, const Geometry &g, const float4 *wtab,
                                      const float *__restrict__ gwt, int p, int j)
{
    __syncwarp();                               // previous read-back done
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        ws.t[p][j][a ^ p] = make_float4(T[0][a].x, T[0][a].y, T[1][a].x, T[1][a].y);
        T[0][a] = T[1][a] = make_float2(0.f, 0.f);
    }
    __syncwarp();
    float4 sum = ws.t[0][j][p];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        const float4 t = ws.t[q][j][p ^ q];
        sum.x += t.x;
        sum.y += t.y;
        sum.z += t.z;
        sum.w += t.w;
    }
    const float4 gw = wtab ? wtab[fw] : __ldg(reinterpret_cast<const float4 *>(gwt) + fw);
    float2 *e0 = sub_s + key + (int64_t)p * g.nz + (int64_t)(2 * j) * g.row_stride;
    float2 *e1 = e0 + g.row_stride;
    atomicAdd(e0, make_float2(sum.x * gw.x, sum.y * gw.x));
    atomicAdd(e0 + 1, make_float2(sum.x * gw.y, sum.y * gw.y));
    atomicAdd(e0 + 2, make_float2(sum.x * gw.z, sum.y * gw.z));
    atomicAdd(e0 + 3, make_float2(sum.x * gw.w, sum.y * gw.w));
    atomicAdd(e1, make_float2(sum.z * gw.x, sum.w * gw.x));
    atomicAdd(e1 + 1, make_float2(sum.z * gw.y, sum.w * gw.y));
    atomicAdd(e1 + 2, make_float2(sum.z * gw.z, sum.w * gw.z));
    atomicAdd(e1 + 3, make_float2(sum.z * gw.w, sum.w * gw.w));
}

// The run state of a warp: T accumulates the run (key, fw) of subgrid s.
struct RunState {
    float2 T[2][8];
    int key, fw, s;             // key -1: no run
    float2 *sub_s;
};

// Accumulates one half batch (32 visibilities, stage S, issued info I,
// values y: lane i holds visibility i's) into the warp's runs.
template <bool T2D>
__device__ __forceinline__ void accumulate_half(RunState &rs, WarpSmem &ws, const RowStage &S, const Issued &I,
                                                float2 yv, const Geometry &g, const float4 *wtab,
                                                const float *__restrict__ gwt, const float *__restrict__ g2,
                                                int p, int j)
{
    if (I.uniform) {
        if (I.key0 != rs.key || I.fw0 != rs.fw) {
            if (rs.key >= 0)
                flush(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
            rs.key = I.key0;
            rs.fw = I.fw0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * k + p;
            float2 y;
            y.x = __shfl_sync(kFull, yv.x, r);
            y.y = __shfl_sync(kFull, yv.y, r);
            accumulate_vis<T2D>(rs.T, S, g2, r, T2D ? __shfl_sync(kFull, I.blk, r) : 0, j, y);
        }
    } else {
        // visibilities in list order; each change of (footprint, w row)
        // ends the run; invalid visibilities (key -1) add nothing
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * k + p;
            const int kr = __shfl_sync(kFull, I.key, r);
            const int fr = __shfl_sync(kFull, I.fw, r);
            const int br = T2D ? __shfl_sync(kFull, I.blk, r) : 0;
            float2 y;
            y.x = __shfl_sync(kFull, yv.x, r);
            y.y = __shfl_sync(kFull, yv.y, r);
            bool done = kr < 0;
#pragma unroll 1
            while (true) {
                const unsigned todo = __ballot_sync(kFull, !done);
                if (todo == 0)
                    break;
                const int leader = __ffs(todo) - 1;
                const int lk = __shfl_sync(kFull, kr, leader);
                const int lf = __shfl_sync(kFull, fr, leader);
                if (lk != rs.key || lf != rs.fw) {
                    if (rs.key >= 0)
                        flush(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
                    rs.key = lk;
                    rs.fw = lf;
                }
                const bool mine = !done && kr == lk && fr == lf;
                accumulate_vis<T2D>(rs.T, S, g2, r, br, j, mine ? y : make_float2(0.f, 0.f));
                done = done || mine;
            }
        }
    }
}

template <bool T2D>
__global__ void __launch_bounds__(kMaxWarps * kWarp, DG_ADJOINT_MIN_BLOCKS)
adjoint_kernel(const Geometry g, const double *__restrict__ uvw, const float2 *__restrict__ vis_in,
               const float *__restrict__ guv, const float *__restrict__ gwt, const Schedule sched,
               float2 *__restrict__ sub_out, DeviceStatus *__restrict__ status,
               const float *__restrict__ g2)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(smem_raw + wtable_bytes(g))[threadIdx.x >> 5];
    const float4 *wtab = load_wtable(g, gwt, smem_raw);
    const int lane = threadIdx.x & 31;
    const int p = lane & 7, j = lane >> 3;

    pdl_wait();                         // the chunk table (and the zeroed output) are complete
    ClaimerT<kStepVis> claimer(sched, lane, Prefetch{uvw, 3 * (int)sizeof(double), vis_in, (int)sizeof(float2)});
    Batch bB = claimer.claim();
    if (bB.n == 0)
        return;
    Issued iB0 = issue_rows<RowStage, !T2D>(half_of(bB, 0), load_uvw(uvw, half_of(bB, 0), lane), g,
                                            ws.st[0][0], guv, lane, status, false);
    Issued iB1 = issue_rows<RowStage, !T2D>(half_of(bB, 1), load_uvw(uvw, half_of(bB, 1), lane), g,
                                            ws.st[0][1], guv, lane, status, true);
    float2 yB0 = load_y(vis_in, half_of(bB, 0), lane), yB1 = load_y(vis_in, half_of(bB, 1), lane);
    Batch bC = claimer.advance(bB);
    Coords3 cC0 = load_uvw(uvw, half_of(bC, 0), lane);
    Coords3 cC1 = load_uvw(uvw, half_of(bC, 1), lane);

    int stage = 0;
    RunState rs;
#pragma unroll
    for (int a = 0; a < 8; ++a)
        rs.T[0][a] = rs.T[1][a] = make_float2(0.f, 0.f);
    rs.key = -1;
    rs.fw = 0;
    rs.s = -1;
    rs.sub_s = sub_out;

    while (bB.n > 0) {
        const Batch bA = bB;
        const Issued iA0 = iB0, iA1 = iB1;
        const float2 yA0 = yB0, yA1 = yB1;
        const int sA = stage;
        bB = bC;
        if (bB.n > 0) {
            iB0 = issue_rows<RowStage, !T2D>(half_of(bB, 0), cC0, g, ws.st[sA ^ 1][0], guv, lane, status,
                                             false);
            iB1 = issue_rows<RowStage, !T2D>(half_of(bB, 1), cC1, g, ws.st[sA ^ 1][1], guv, lane, status,
                                             true);
            yB0 = load_y(vis_in, half_of(bB, 0), lane);
            yB1 = load_y(vis_in, half_of(bB, 1), lane);
        }
        bC = claimer.advance(bC);
        cC0 = load_uvw(uvw, half_of(bC, 0), lane);
        cC1 = load_uvw(uvw, half_of(bC, 1), lane);
        if (bB.n > 0)
            cp_async_wait<1>();
        else
            cp_async_wait<0>();
        __syncwarp();

        if (bA.s != rs.s) {
            if (rs.key >= 0)
                flush(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
            rs.key = -1;
            rs.s = bA.s;
            rs.sub_s = sub_out + (int64_t)bA.s * g.plane;
        }
        accumulate_half<T2D>(rs, ws, ws.st[sA][0], iA0, yA0, g, wtab, gwt, g2, p, j);
        if (bA.n > kBatch)
            accumulate_half<T2D>(rs, ws, ws.st[sA][1], iA1, yA1, g, wtab, gwt, g2, p, j);
        __syncwarp();
        stage ^= 1;
    }
    if (rs.key >= 0)
        flush(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
}

size_t smem_bytes(const degrid_plan *p)
{
    return wtable_bytes_host(p->geo) + sizeof(WarpSmem) * (size_t)p->warps_per_block;
}

// Dynamic shared memory opened so far for the plan's kernel instance on its device.
std::atomic<size_t> &smem_record(const degrid_plan *p)
{
    static std::atomic<size_t> table[2][kMaxDevices];
    return dg_smem_record(table[p->guv2 ? 1 : 0], p->device);
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
    auto kernel = p->guv2 ? adjoint_kernel<true> : adjoint_kernel<false>;
    const cudaError_t e = dg_open_smem(smem_record(p), kernel, smem);
    if (e != cudaSuccess)
        return e;
    return launch_pdl(kernel, dim3(grid_blocks), dim3(p->warps_per_block * kWarp), smem, st, p->geo, uvw,
                      reinterpret_cast<const float2 *>(vis_in), (const float *)p->guv, (const float *)p->gw,
                      sched, reinterpret_cast<float2 *>(sub_out), p->status, (const float *)p->guv2);
}

int dg_max_blocks_per_sm_adjoint(degrid_plan *p)
{
    using namespace dg;
    int n = 0;
    const size_t smem = smem_bytes(p);
    auto kernel = p->guv2 ? adjoint_kernel<true> : adjoint_kernel<false>;
    if (dg_open_smem(smem_record(p), kernel, smem) != cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, p->warps_per_block * kWarp, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}
