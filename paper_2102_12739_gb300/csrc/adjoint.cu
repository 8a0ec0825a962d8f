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
// 8j + p adds column a = p of rows 2j, 2j+1 to the subgrid: the four w
// planes c = 0..3 of an element are 32 contiguous bytes, two 16-byte vector
// reductions (red.global.add.v4.f32) when nz = 4 and the output is 16-byte
// aligned, else four float2 atomics.  Dense lists have runs of hundreds of
// visibilities, so the adds are a small fraction of the work.  Halves whose
// 32 visibilities share one run take a branch-free path.
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

// This lane's stage reads in pass 0 of a half; pass k reads row 8k + p, 8 rows
// (16 float4 of u, 32 float2 of v) further on.  The slot swizzle of row
// 8k + p is that of row p (bit 2 of the row is bit 2 of p).
struct LaneRows {
    const float4 *u0, *u1;
    const float2 *v;
};

__device__ __forceinline__ LaneRows lane_rows(const RowStage &S, int p, int j)
{
    const int sw = (p >> 2) & 1;
    return {&S.u[p][sw], &S.u[p][sw ^ 1], reinterpret_cast<const float2 *>(&S.v[p][(j >> 1) ^ sw]) + (j & 1)};
}

// T[i][a] += g_u[a] * (g_v[2j + i] * y) for the visibility of pass k.
__device__ __forceinline__ void accumulate(float2 (&T)[2][8], const LaneRows &L, int k, float2 y)
{
    const float4 u0 = L.u0[16 * k];
    const float4 u1 = L.u1[16 * k];
    const float2 v = L.v[32 * k];
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
__device__ __forceinline__ void accumulate_vis(float2 (&T)[2][8], const LaneRows &L,
                                               const float *__restrict__ g2, int k, int blk, int j,
                                               float2 y)
{
    if (T2D)
        accumulate_2d(T, g2, blk, j, y);
    else
        accumulate(T, L, k, y);
}

// Adds the run (key, fw) to the subgrid at sub_s and clears T.  kVec4: every
// element's four w planes start on a 16-byte boundary (nz = 4, so z0 = 0, and
// an aligned output), added as two float4 reductions.
template <bool kVec4>
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
    const float4 t0 = ws.t[0][j][p];
    float2 s0 = make_float2(t0.x, t0.y), s1 = make_float2(t0.z, t0.w);     // T[2j][p], T[2j+1][p]
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        const float4 t = ws.t[q][j][p ^ q];
        s0 = __fadd2_rn(s0, make_float2(t.x, t.y));
        s1 = __fadd2_rn(s1, make_float2(t.z, t.w));
    }
    const float4 gw = wtab ? wtab[fw] : __ldg(reinterpret_cast<const float4 *>(gwt) + fw);
    float2 *e0 = sub_s + key + (int64_t)p * g.nz + (int64_t)(2 * j) * g.row_stride;
    float2 *e1 = e0 + g.row_stride;
    const float gc[4] = {gw.x, gw.y, gw.z, gw.w};
    if (kVec4) {
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            const float2 a0 = __fmul2_rn(s0, make_float2(gc[c], gc[c]));
            const float2 a1 = __fmul2_rn(s0, make_float2(gc[c + 1], gc[c + 1]));
            const float2 b0 = __fmul2_rn(s1, make_float2(gc[c], gc[c]));
            const float2 b1 = __fmul2_rn(s1, make_float2(gc[c + 1], gc[c + 1]));
            atomicAdd(reinterpret_cast<float4 *>(e0 + c), make_float4(a0.x, a0.y, a1.x, a1.y));
            atomicAdd(reinterpret_cast<float4 *>(e1 + c), make_float4(b0.x, b0.y, b1.x, b1.y));
        }
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            atomicAdd(e0 + c, __fmul2_rn(s0, make_float2(gc[c], gc[c])));
            atomicAdd(e1 + c, __fmul2_rn(s1, make_float2(gc[c], gc[c])));
        }
    }
}

// The run state of a warp: T accumulates the run (key, fw) of subgrid s.
struct RunState {
    float2 T[2][8];
    int key, fw, s;             // key -1: no run
    float2 *sub_s;
};

// Accumulates one half batch (32 visibilities, stage S, issued info I,
// values y: lane i holds visibility i's) into the warp's runs.
template <bool T2D, bool kVec4>
__device__ __forceinline__ void accumulate_half(RunState &rs, WarpSmem &ws, const RowStage &S, const Issued &I,
                                                float2 yv, const Geometry &g, const float4 *wtab,
                                                const float *__restrict__ gwt, const float *__restrict__ g2,
                                                int p, int j)
{
    const LaneRows L = lane_rows(S, p, j);
    if (I.uniform) {
        if (I.key0 != rs.key || I.fw0 != rs.fw) {
            if (rs.key >= 0)
                flush<kVec4>(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
            rs.key = I.key0;
            rs.fw = I.fw0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * k + p;
            float2 y;
            y.x = __shfl_sync(kFull, yv.x, r);
            y.y = __shfl_sync(kFull, yv.y, r);
            accumulate_vis<T2D>(rs.T, L, g2, k, T2D ? __shfl_sync(kFull, I.blk, r) : 0, j, y);
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
                        flush<kVec4>(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
                    rs.key = lk;
                    rs.fw = lf;
                }
                const bool mine = !done && kr == lk && fr == lf;
                accumulate_vis<T2D>(rs.T, L, g2, k, br, j, mine ? y : make_float2(0.f, 0.f));
                done = done || mine;
            }
        }
    }
}

template <bool T2D, bool kVec4>
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
                flush<kVec4>(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
            rs.key = -1;
            rs.s = bA.s;
            rs.sub_s = sub_out + (int64_t)bA.s * g.plane;
        }
        accumulate_half<T2D, kVec4>(rs, ws, ws.st[sA][0], iA0, yA0, g, wtab, gwt, g2, p, j);
        if (bA.n > kBatch)
            accumulate_half<T2D, kVec4>(rs, ws, ws.st[sA][1], iA1, yA1, g, wtab, gwt, g2, p, j);
        __syncwarp();
        stage ^= 1;
    }
    if (rs.key >= 0)
        flush<kVec4>(rs.T, ws, rs.sub_s, rs.key, rs.fw, g, wtab, gwt, p, j);
}

size_t smem_bytes(const degrid_plan *p)
{
    return wtable_bytes_host(p->geo) + sizeof(WarpSmem) * (size_t)p->warps_per_block;
}

// The kernel instance for a 2D table (or not) and vector reductions (or not).
using AdjointKernel = decltype(&adjoint_kernel<false, false>);

AdjointKernel kernel_for(const degrid_plan *p, bool vec4)
{
    if (p->guv2)
        return vec4 ? adjoint_kernel<true, true> : adjoint_kernel<true, false>;
    return vec4 ? adjoint_kernel<false, true> : adjoint_kernel<false, false>;
}

// Vector reductions need every element's 32 bytes of w planes 16-byte
// aligned: nz = kW (so z0 = 0 and every element index is a multiple of 4)
// and a 16-byte aligned output.
bool vec4_ok(const degrid_plan *p, const void *sub_out)
{
    return p->geo.nz == kW && (reinterpret_cast<uintptr_t>(sub_out) & 15u) == 0;
}

// Dynamic shared memory opened so far for the plan's kernel instance on its device.
std::atomic<size_t> &smem_record(const degrid_plan *p, bool vec4)
{
    static std::atomic<size_t> table[4][kMaxDevices];
    return dg_smem_record(table[(p->guv2 ? 2 : 0) + (vec4 ? 1 : 0)], p->device);
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
    const bool vec4 = vec4_ok(p, sub_out);
    const AdjointKernel kernel = kernel_for(p, vec4);
    const cudaError_t e = dg_open_smem(smem_record(p, vec4), kernel, smem);
    if (e != cudaSuccess)
        return e;
    return launch_pdl(kernel, dim3(grid_blocks), dim3(p->warps_per_block * kWarp), smem, st, p->geo, uvw,
                      reinterpret_cast<const float2 *>(vis_in), (const float *)p->guv, (const float *)p->gw,
                      sched, reinterpret_cast<float2 *>(sub_out), p->status, (const float *)p->guv2);
}

// Resident CTAs per SM of the instance an aligned output would run (both
// instances have the same launch bounds and shared memory).
int dg_max_blocks_per_sm_adjoint(degrid_plan *p)
{
    using namespace dg;
    int n = 0;
    const size_t smem = smem_bytes(p);
    const bool vec4 = p->geo.nz == kW;
    const AdjointKernel kernel = kernel_for(p, vec4);
    if (dg_open_smem(smem_record(p, vec4), kernel, smem) != cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, p->warps_per_block * kWarp, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}
