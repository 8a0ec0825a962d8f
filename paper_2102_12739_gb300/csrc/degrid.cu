// Degridding kernel (paper Section "Implementation": kernel D1 and its
// variants), re-designed for sm_103a.
//
// Work decomposition (pipeline.cuh).  A persistent grid of warps walks chunks
// of consecutive visibilities of one subgrid in steps of 64 (two halves of
// 32, which amortises the per-step bookkeeping and gives every lane two
// independent coordinates to snap).  Three stages overlap across consecutive
// steps of a warp:
//  1. the FP64 coordinates of step n + 2 are loaded into registers (and the
//     next chunk's are prefetched into L2 when its descriptor arrives);
//  2. step n + 1 is snapped (one visibility per lane and half) and its g_u and
//     g_v rows are copied into the warp's shared-memory stage with cp.async;
//  3. step n is summed from the stage that arrived, one half after the other.
//
// Footprint sum.  The separable weights let the 8 x 8 x 4 sum be taken in
// three contractions,
//     V = sum_b g_v[b] sum_a g_u[a] M[b][a],   M[b][a] = sum_c g_w[c] s[y0+b][x0+a][z0+c],
// and M depends only on the footprint start and the w-kernel row.  On a dense
// list hundreds of consecutive visibilities share both (the reuse the paper
// notes for D1), so M is computed once per run and each visibility then costs
// 72 complex x real products instead of 256.
//
// Lanes.  Four lanes share a visibility: lane 8j + p (j = 0..3, p = 0..7)
// holds the rows M[2j][0..7] and M[2j+1][0..7] of the footprint in 32
// registers and, for a visibility r, forms
// sum_{b = 2j, 2j+1} g_v[b] sum_a g_u[a] M[b][a] (36 FP32 operations).  A
// half takes four passes; in pass k lane 8j + p works on visibility
// 8 (k ^ j) + p, an order chosen so that the two exchange steps of the
// reduction move the same pass slots on every lane (no selects): lane xor 16
// adds slots 2, 3 to 0, 1, then lane xor 8 adds slot 1 to slot 0, and lane
// 8j + p ends with visibility 8j + p, so the warp writes its 32 results into
// one contiguous 256-byte segment in lane order.  The 8 lanes of one 128-bit
// shared-memory wavefront read 8 consecutive rows of the stage, which its
// half-swapped layout places in 8 different bank groups.  M is built by the
// whole warp (two entries per lane) into shared memory and read back by rows;
// a half whose 32 visibilities share one footprint and w row needs no checks,
// and any other half is summed once per distinct (footprint, w row) it holds,
// every lane keeping the pass that matches its own visibility.
// The products use packed FFMA2 on (re, im) pairs with a duplicated real
// weight: bitwise the same as two scalar FMAs, in half the instructions
// (11.2 instead of 12.7 warp instructions per visibility on dense lines).
#include "pipeline.cuh"

namespace dg {
namespace {

#ifndef DG_DEGRID_MIN_BLOCKS
#define DG_DEGRID_MIN_BLOCKS 2   // resident CTAs per SM the register budget is sized for
#endif

constexpr int kMaxWarps = 8;                // per CTA
constexpr int kBatchVis = 2 * kBatch;       // visibilities per pipeline step (two halves)
struct alignas(128) WarpSmem {
    RowStage st[2][2];          // [stage][half]
    float2 m[8][8];             // M[b][a] of the footprint being built
    float2 part[4][kWarp];      // per-pass partials on the mixed path
};

// ---- the factored sum -------------------------------------------------------

// M[2j + i][a] for i = 0, 1 and a = 0..7 of footprint `key` (subgrid at
// `base`) with w row gw: lane (a = lane & 7, b = lane >> 3 and b + 4)
// computes two entries into shared memory, then every lane reads its rows.
// sum_c g_w[c] s[e + c] for one footprint point (the entries of M; the
// direct arm forms them the same way, so both arms round alike).
// With `vec` (16-byte aligned subgrids, nz a multiple of the elements per
// 16 bytes, and a footprint start z0 that is one too) the four elements are
// read with 16-byte loads.
template <int DT>
__device__ __forceinline__ float2 footprint_point(const void *sub, int64_t e, const float4 &gw, bool vec)
{
    float2 s[4];
    if (vec) {
        Storage<DT>::load4(sub, e, s);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
            s[c] = Storage<DT>::load(sub, e + c);
    }
    float2 m;
    m.x = fmaf(s[3].x, gw.w, fmaf(s[2].x, gw.z, fmaf(s[1].x, gw.y, s[0].x * gw.x)));
    m.y = fmaf(s[3].y, gw.w, fmaf(s[2].y, gw.z, fmaf(s[1].y, gw.y, s[0].y * gw.x)));
    return m;
}

// Whether the footprint starting at `key` can use 16-byte loads.
template <int DT>
__device__ __forceinline__ bool vec_footprint(bool vec_ok, int key)
{
    return vec_ok && (key % Storage<DT>::kQuad) == 0;
}

template <int DT>
__device__ __forceinline__ void build_rows(float2 (&M)[2][8], float2 (&mbuf)[8][8], const void *sub,
                                           int64_t base, int key, const float4 &gw, const Geometry &g,
                                           bool vec_ok, int lane, int j)
{
    const int a = lane & 7, b = lane >> 3;
    const int64_t col = base + key + (int64_t)a * g.nz;
    const bool vec = vec_footprint<DT>(vec_ok, key);
    __syncwarp();                               // previous read-back done
#pragma unroll
    for (int k = 0; k < 2; ++k)
        mbuf[b + 4 * k][a] = footprint_point<DT>(sub, col + (int64_t)(b + 4 * k) * g.row_stride, gw, vec);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int a2 = 0; a2 < 8; a2 += 2) {
            const float4 t = *reinterpret_cast<const float4 *>(&mbuf[2 * j + i][a2]);
            M[i][a2] = make_float2(t.x, t.y);
            M[i][a2 + 1] = make_float2(t.z, t.w);
        }
    }
}

// This lane's quarter of visibility r: sum_{i} g_v[2j + i] sum_a g_u[a] M[i][a].
__device__ __forceinline__ float2 quarter_sum(const float2 (&M)[2][8], const RowStage &S, int r, int j)
{
    const float4 u0 = S.u[r][row_half(r, 0)];
    const float4 u1 = S.u[r][row_half(r, 1)];
    const float2 v = reinterpret_cast<const float2 *>(&S.v[r][row_half(r, j >> 1)])[j & 1];
    const float gu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    // complex x real products as packed pairs (re, im) * (g, g): one FFMA2
    // per product, each half rounded exactly as a scalar FMA
    float2 t0 = __fmul2_rn(M[0][0], make_float2(gu[0], gu[0]));
    float2 t1 = __fmul2_rn(M[1][0], make_float2(gu[0], gu[0]));
#pragma unroll
    for (int a = 1; a < 8; ++a) {
        t0 = __ffma2_rn(M[0][a], make_float2(gu[a], gu[a]), t0);
        t1 = __ffma2_rn(M[1][a], make_float2(gu[a], gu[a]), t1);
    }
    return __ffma2_rn(t1, make_float2(v.y, v.y), __fmul2_rn(t0, make_float2(v.x, v.x)));
}

// 2D G_uv table: this lane's quarter sum_{i} sum_a G[blk][2j + i][a] M[i][a]
// with the 16 weights of rows 2j, 2j + 1 of the visibility's block read
// straight from the (L2-resident) table.
__device__ __forceinline__ float2 quarter_sum_2d(const float2 (&M)[2][8], const float *__restrict__ g2,
                                                 int blk, int j)
{
    const float4 *w = reinterpret_cast<const float4 *>(g2 + (size_t)blk * (kUV * kUV) + 2 * kUV * j);
    const float4 w0 = __ldg(w), w1 = __ldg(w + 1), w2 = __ldg(w + 2), w3 = __ldg(w + 3);
    const float g0[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    const float g1[8] = {w2.x, w2.y, w2.z, w2.w, w3.x, w3.y, w3.z, w3.w};
    float2 t0 = __fmul2_rn(M[0][0], make_float2(g0[0], g0[0]));
    float2 t1 = __fmul2_rn(M[1][0], make_float2(g1[0], g1[0]));
#pragma unroll
    for (int a = 1; a < 8; ++a) {
        t0 = __ffma2_rn(M[0][a], make_float2(g0[a], g0[a]), t0);
        t1 = __ffma2_rn(M[1][a], make_float2(g1[a], g1[a]), t1);
    }
    return __fadd2_rn(t0, t1);
}

// One pass: the separable sum from the staged rows, or the 2D table sum.
template <bool T2D>
__device__ __forceinline__ float2 pass_sum(const float2 (&M)[2][8], const RowStage &S,
                                           const float *__restrict__ g2, int r, int blk, int j)
{
    return T2D ? quarter_sum_2d(M, g2, blk, j) : quarter_sum(M, S, r, j);
}

// Direct arm: this lane's quarter of visibility r (footprint `key`, w row gw)
// from the subgrid itself, M's two rows formed on the fly; the same
// operations in the same order as build_rows followed by quarter_sum.
template <int DT>
__device__ __forceinline__ float2 quarter_sum_direct(const void *sub, int64_t base, int key,
                                                    const float4 &gw, const RowStage &S, int r, int j,
                                                    const Geometry &g, bool vec_ok)
{
    const bool vec = vec_footprint<DT>(vec_ok, key);
    const float4 u0 = S.u[r][row_half(r, 0)];
    const float4 u1 = S.u[r][row_half(r, 1)];
    const float2 v = reinterpret_cast<const float2 *>(&S.v[r][row_half(r, j >> 1)])[j & 1];
    const float gu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    const int64_t e0 = base + key + (int64_t)(2 * j) * g.row_stride, e1 = e0 + g.row_stride;
    float2 m0[8], m1[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {             // all loads issued before the sums
        m0[a] = footprint_point<DT>(sub, e0 + (int64_t)a * g.nz, gw, vec);
        m1[a] = footprint_point<DT>(sub, e1 + (int64_t)a * g.nz, gw, vec);
    }
    float2 t0 = __fmul2_rn(m0[0], make_float2(gu[0], gu[0]));
    float2 t1 = __fmul2_rn(m1[0], make_float2(gu[0], gu[0]));
#pragma unroll
    for (int a = 1; a < 8; ++a) {
        t0 = __ffma2_rn(m0[a], make_float2(gu[a], gu[a]), t0);
        t1 = __ffma2_rn(m1[a], make_float2(gu[a], gu[a]), t1);
    }
    return __ffma2_rn(t1, make_float2(v.y, v.y), __fmul2_rn(t0, make_float2(v.x, v.x)));
}

// Error-free sum (Knuth's TwoSum): a + b = s + e exactly, s = fl(a + b).
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// State of the cached footprint matrix: rows 2j, 2j + 1 of M for (key, fw)
// in the subgrid at `base` (key -2: none).
struct MState {
    float2 M[2][8];
    int key, fw;
};

// Sums one half batch (32 visibilities, stage S, issued info I), reduces the
// four lane partials and stores visibility `lane` of the half.
// Reduces the four pass slots of every lane to visibility `lane` of the half
// and stores it (times the subgrid's scale for FP16/BF16 storage).
template <int DT, bool COMP>
__device__ __forceinline__ void reduce_store(float2 (&P)[4], const Batch &h, float sc,
                                             float2 *__restrict__ vis_out, int lane)
{
    // lane xor 16 (j ^ 2) brings slots 2, 3 onto 0, 1; lane xor 8 (j ^ 1)
    // brings slot 1 onto 0
    float2 V;
    if (COMP) {
        // the same three additions as error-free sums; the four rounding
        // errors are summed and added back once
        float2 e0, e1, e;
        P[0].x = two_sum(P[0].x, __shfl_xor_sync(kFull, P[2].x, 16), e0.x);
        P[0].y = two_sum(P[0].y, __shfl_xor_sync(kFull, P[2].y, 16), e0.y);
        P[1].x = two_sum(P[1].x, __shfl_xor_sync(kFull, P[3].x, 16), e1.x);
        P[1].y = two_sum(P[1].y, __shfl_xor_sync(kFull, P[3].y, 16), e1.y);
        V.x = two_sum(P[0].x, __shfl_xor_sync(kFull, P[1].x, 8), e.x);
        V.y = two_sum(P[0].y, __shfl_xor_sync(kFull, P[1].y, 8), e.y);
        e.x += e0.x + __shfl_xor_sync(kFull, e1.x, 8);
        e.y += e0.y + __shfl_xor_sync(kFull, e1.y, 8);
        V.x += e.x;
        V.y += e.y;
    } else {
        P[0].x += __shfl_xor_sync(kFull, P[2].x, 16);
        P[0].y += __shfl_xor_sync(kFull, P[2].y, 16);
        P[1].x += __shfl_xor_sync(kFull, P[3].x, 16);
        P[1].y += __shfl_xor_sync(kFull, P[3].y, 16);
        V.x = P[0].x + __shfl_xor_sync(kFull, P[1].x, 8);
        V.y = P[0].y + __shfl_xor_sync(kFull, P[1].y, 8);
    }
    if (DT != DG_C64)
        V = __fmul2_rn(V, make_float2(sc, sc));
    if (lane < h.n)                     // lane 8j + p holds visibility 8j + p of the half
        vis_out[h.b0 + lane] = V;
}


template <int DT, bool COMP, bool DIRECT, bool T2D>
__device__ __forceinline__ void sum_half(MState &ms, WarpSmem &ws, const RowStage &S, const Issued &I,
                                         const Batch &h, const void *__restrict__ subgrids, int64_t base,
                                         float sc, const Geometry &g, const float4 *wtab,
                                         const float *__restrict__ gwt, float2 *__restrict__ vis_out,
                                         int direct_runs, bool vec_ok, const float *__restrict__ g2,
                                         int lane, int p, int j)
{
    float2 P[4];                        // pass k: this lane's quarter of visibility 8 (k ^ j) + p
    if (I.uniform) {
        if (I.key0 != ms.key || I.fw0 != ms.fw) {
            const float4 gw = wtab ? wtab[I.fw0] : __ldg(reinterpret_cast<const float4 *>(gwt) + I.fw0);
            build_rows<DT>(ms.M, ws.m, subgrids, base, I.key0, gw, g, vec_ok, lane, j);
            ms.key = I.key0;
            ms.fw = I.fw0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * (k ^ j) + p;
            P[k] = pass_sum<T2D>(ms.M, S, g2, r, T2D ? __shfl_sync(kFull, I.blk, r) : 0, j);
        }
    } else if (DIRECT && !T2D && I.runs >= direct_runs) {
        // Short runs: every visibility is summed from its own footprint
        // (pass k covers visibilities 8k .. 8k + 7; invalid ones stay zero).
        // Pays off when the footprints of a half overlap (slowly moving
        // lists whose w row changes often: the other visibilities keep them
        // in L1); for footprints scattered over the subgrid the cooperative
        // M builds below read it in longer contiguous pieces and win.  A
        // separate kernel instance, so the register budget of the plain
        // path is untouched.
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * k + p;
            const int kr = __shfl_sync(kFull, I.key, r);
            const int fr = __shfl_sync(kFull, I.fw, r);
            float2 acc = make_float2(0.f, 0.f);
            if (kr >= 0) {
                const float4 gw = wtab ? wtab[fr] : __ldg(reinterpret_cast<const float4 *>(gwt) + fr);
                acc = quarter_sum_direct<DT>(subgrids, base, kr, gw, S, r, j, g, vec_ok);
            }
            ws.part[k][lane] = acc;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k)
            P[k] = ws.part[k ^ j][lane];
        __syncwarp();
    } else {
        // Pass k covers visibilities 8k .. 8k + 7 here, so a change of
        // footprint inside a run of the list touches one pass.  Each pass is
        // summed once per distinct (footprint, w row) among its visibilities,
        // every lane keeping the sum that matches its own (invalid ones, key
        // -1, stay zero); the partials then move to the slots of the permuted
        // order, slot k = pass k ^ j.
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            const int r = 8 * k + p;
            const int kr = __shfl_sync(kFull, I.key, r);
            const int fr = __shfl_sync(kFull, I.fw, r);
            bool done = kr < 0;
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll 1
            while (true) {
                const unsigned todo = __ballot_sync(kFull, !done);
                if (todo == 0)
                    break;
                const int leader = __ffs(todo) - 1;
                const int lk = __shfl_sync(kFull, kr, leader);
                const int lf = __shfl_sync(kFull, fr, leader);
                if (lk != ms.key || lf != ms.fw) {
                    const float4 gw = wtab ? wtab[lf] : __ldg(reinterpret_cast<const float4 *>(gwt) + lf);
                    build_rows<DT>(ms.M, ws.m, subgrids, base, lk, gw, g, vec_ok, lane, j);
                    ms.key = lk;
                    ms.fw = lf;
                }
                const float2 x = pass_sum<T2D>(ms.M, S, g2, r, T2D ? __shfl_sync(kFull, I.blk, r) : 0, j);
                const bool mine = !done && kr == lk && fr == lf;
                if (mine)
                    acc = x;
                done = done || mine;
            }
            ws.part[k][lane] = acc;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 4; ++k)
            P[k] = ws.part[k ^ j][lane];
        __syncwarp();
    }
    reduce_store<DT, COMP>(P, h, sc, vis_out, lane);
}

// Both halves of a full step share one footprint and w row (the common
// case on dense lists): their eight passes are summed in one block, so the
// scheduler can interleave the two halves' loads and FMA chains.
template <int DT, bool COMP, bool T2D>
__device__ __forceinline__ void sum_step_uniform(MState &ms, WarpSmem &ws, const RowStage &S0,
                                                 const RowStage &S1, const Issued &I0, const Issued &I1,
                                                 const Batch &b, const void *__restrict__ subgrids,
                                                 int64_t base, float sc, const Geometry &g,
                                                 const float4 *wtab, const float *__restrict__ gwt,
                                                 float2 *__restrict__ vis_out, bool vec_ok,
                                                 const float *__restrict__ g2, int lane, int p, int j)
{
    if (I0.key0 != ms.key || I0.fw0 != ms.fw) {
        const float4 gw = wtab ? wtab[I0.fw0] : __ldg(reinterpret_cast<const float4 *>(gwt) + I0.fw0);
        build_rows<DT>(ms.M, ws.m, subgrids, base, I0.key0, gw, g, vec_ok, lane, j);
        ms.key = I0.key0;
        ms.fw = I0.fw0;
    }
    float2 P0[4], P1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = 8 * (k ^ j) + p;
        P0[k] = pass_sum<T2D>(ms.M, S0, g2, r, T2D ? __shfl_sync(kFull, I0.blk, r) : 0, j);
        P1[k] = pass_sum<T2D>(ms.M, S1, g2, r, T2D ? __shfl_sync(kFull, I1.blk, r) : 0, j);
    }
    reduce_store<DT, COMP>(P0, half_of(b, 0), sc, vis_out, lane);
    reduce_store<DT, COMP>(P1, half_of(b, 1), sc, vis_out, lane);
}

template <int DT, bool COMP, bool DIRECT, bool T2D>
__global__ void __launch_bounds__(kMaxWarps * kWarp, DG_DEGRID_MIN_BLOCKS)
degrid_kernel(const Geometry g, const void *__restrict__ subgrids, const float *__restrict__ scale,
              const double *__restrict__ uvw, const float *__restrict__ guv,
              const float *__restrict__ gwt, const Schedule sched, float2 *__restrict__ vis_out,
              DeviceStatus *__restrict__ status, const int direct_runs, const bool vec_ok,
              const float *__restrict__ g2, const bool prefetch_uvw)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // [w table (optional)] [one WarpSmem per warp]
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(smem_raw + wtable_bytes(g))[threadIdx.x >> 5];
    const float4 *wtab = load_wtable(g, gwt, smem_raw);
    const int lane = threadIdx.x & 31;
    const int p = lane & 7, j = lane >> 3;

    // coordinates in device memory are prefetched into L2 a chunk ahead;
    // coordinates read in place from host memory are not (the host link
    // bounds those calls, and one batch of lead hides its latency)
    pdl_wait();                         // the chunk table is complete
    ClaimerT<kBatchVis> claimer(sched, lane,
                                Prefetch{prefetch_uvw ? uvw : nullptr, 3 * (int)sizeof(double), nullptr, 0});
    Batch bB = claimer.claim();         // rows in flight
    if (bB.n == 0)
        return;
    Issued iB0 = issue_rows<RowStage, !T2D>(half_of(bB, 0), load_uvw(uvw, half_of(bB, 0), lane), g,
                                            ws.st[0][0], guv, lane, status, false);
    Issued iB1 = issue_rows<RowStage, !T2D>(half_of(bB, 1), load_uvw(uvw, half_of(bB, 1), lane), g,
                                            ws.st[0][1], guv, lane, status, true);
    Batch bC = claimer.advance(bB);     // coordinates in registers
    Coords3 cC0 = load_uvw(uvw, half_of(bC, 0), lane);
    Coords3 cC1 = load_uvw(uvw, half_of(bC, 1), lane);

    int stage = 0;
    MState ms;
    ms.key = -2;
    ms.fw = -1;
    int m_s = -1;
    int64_t base = 0;
    float sc = 1.f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int a = 0; a < 8; ++a)
            ms.M[i][a] = make_float2(0.f, 0.f);

    while (bB.n > 0) {
        const Batch bA = bB;            // summed in this iteration
        const Issued iA0 = iB0, iA1 = iB1;
        const int sA = stage;
        bB = bC;
        if (bB.n > 0) {
            iB0 = issue_rows<RowStage, !T2D>(half_of(bB, 0), cC0, g, ws.st[sA ^ 1][0], guv, lane, status,
                                             false);
            iB1 = issue_rows<RowStage, !T2D>(half_of(bB, 1), cC1, g, ws.st[sA ^ 1][1], guv, lane, status,
                                             true);
        }
        bC = claimer.advance(bC);
        cC0 = load_uvw(uvw, half_of(bC, 0), lane);
        cC1 = load_uvw(uvw, half_of(bC, 1), lane);
        if (bB.n > 0)
            cp_async_wait<1>();         // the stage of batch A; batch B may stay in flight
        else
            cp_async_wait<0>();
        __syncwarp();

        if (bA.s != m_s) {
            m_s = bA.s;
            ms.key = -2;
            base = (int64_t)bA.s * g.plane;
            if (DT != DG_C64)
                sc = __ldg(scale + bA.s);
        }
        if (iA0.uniform && iA1.uniform && iA0.key0 == iA1.key0 && iA0.fw0 == iA1.fw0 &&
            bA.n == kBatchVis) {
            sum_step_uniform<DT, COMP, T2D>(ms, ws, ws.st[sA][0], ws.st[sA][1], iA0, iA1, bA, subgrids,
                                            base, sc, g, wtab, gwt, vis_out, vec_ok, g2, lane, p, j);
        } else {
            sum_half<DT, COMP, DIRECT, T2D>(ms, ws, ws.st[sA][0], iA0, half_of(bA, 0), subgrids, base, sc,
                                            g, wtab, gwt, vis_out, direct_runs, vec_ok, g2, lane, p, j);
            if (bA.n > kBatch)
                sum_half<DT, COMP, DIRECT, T2D>(ms, ws, ws.st[sA][1], iA1, half_of(bA, 1), subgrids, base,
                                                sc, g, wtab, gwt, vis_out, direct_runs, vec_ok, g2, lane,
                                                p, j);
        }
        __syncwarp();
        stage ^= 1;
    }
}

size_t smem_bytes(const degrid_plan *p, int warps)
{
    return wtable_bytes_host(p->geo) + sizeof(WarpSmem) * (size_t)warps;
}

// Dynamic shared memory opened so far for a kernel instance on a device.
template <int DT, bool COMP, bool DIRECT, bool T2D>
std::atomic<size_t> &smem_record(int device)
{
    static std::atomic<size_t> table[kMaxDevices];
    return dg_smem_record(table, device);
}

template <int DT, bool COMP, bool DIRECT, bool T2D>
cudaError_t launch(degrid_plan *p, cudaStream_t st, const void *subgrids, const float *scale,
                   const double *uvw, float2 *out, const Schedule &sched, int grid_blocks)
{
    const int threads = p->warps_per_block * kWarp;
    const size_t smem = smem_bytes(p, p->warps_per_block);
    cudaError_t e = dg_open_smem(smem_record<DT, COMP, DIRECT, T2D>(p->device), degrid_kernel<DT, COMP, DIRECT, T2D>,
                                 smem);
    if (e != cudaSuccess)
        return e;
    // 16-byte footprint loads need an aligned stack and nz a multiple of the
    // elements per 16 bytes
    const bool vec_ok = (reinterpret_cast<uintptr_t>(subgrids) & 15) == 0 &&
                        p->geo.nz % Storage<DT>::kQuad == 0;
    return launch_pdl(degrid_kernel<DT, COMP, DIRECT, T2D>, dim3(grid_blocks), dim3(threads), smem, st,
                      p->geo, subgrids, scale, uvw, (const float *)p->guv, (const float *)p->gw, sched, out,
                      p->status, p->direct_runs, vec_ok, (const float *)p->guv2, !p->host_inputs);
}

template <int DT, bool COMP, bool DIRECT, bool T2D>
int max_blocks(degrid_plan *p)
{
    int n = 0;
    const size_t smem = smem_bytes(p, p->warps_per_block);
    if (dg_open_smem(smem_record<DT, COMP, DIRECT, T2D>(p->device), degrid_kernel<DT, COMP, DIRECT, T2D>, smem) !=
        cudaSuccess)
        return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, degrid_kernel<DT, COMP, DIRECT, T2D>,
                                                      p->warps_per_block * kWarp, smem) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

// Kernel instance of a plan: storage type, compensated reduction, and one of
// three summing forms (footprint cache; with the direct arm; 2D G_uv table).
template <int DT, bool COMP>
cudaError_t launch_form(degrid_plan *p, cudaStream_t st, const void *subgrids, const float *scale,
                        const double *uvw, float2 *out, const Schedule &sched, int grid_blocks)
{
    if (p->guv2)
        return launch<DT, COMP, false, true>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    if (p->direct_runs < DG_DIRECT_RUNS_NEVER)
        return launch<DT, COMP, true, false>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    return launch<DT, COMP, false, false>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
}

template <int DT, bool COMP>
int max_blocks_form(degrid_plan *p)
{
    if (p->guv2)
        return max_blocks<DT, COMP, false, true>(p);
    if (p->direct_runs < DG_DIRECT_RUNS_NEVER)
        return max_blocks<DT, COMP, true, false>(p);
    return max_blocks<DT, COMP, false, false>(p);
}

template <int DT>
cudaError_t launch_dt(degrid_plan *p, cudaStream_t st, const void *subgrids, const float *scale,
                      const double *uvw, float2 *out, const Schedule &sched, int grid_blocks)
{
    return p->compensated ? launch_form<DT, true>(p, st, subgrids, scale, uvw, out, sched, grid_blocks)
                          : launch_form<DT, false>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
}

template <int DT>
int max_blocks_dt(degrid_plan *p)
{
    return p->compensated ? max_blocks_form<DT, true>(p) : max_blocks_form<DT, false>(p);
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
        return launch_dt<DG_C64>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    case DG_C32_F16:
        return launch_dt<DG_C32_F16>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    case DG_C32_BF16:
        return launch_dt<DG_C32_BF16>(p, st, subgrids, scale, uvw, out, sched, grid_blocks);
    }
    return cudaErrorInvalidValue;
}

int dg_max_blocks_per_sm_degrid(degrid_plan *p)
{
    using namespace dg;
    switch (p->dtype) {
    case DG_C64: return max_blocks_dt<DG_C64>(p);
    case DG_C32_F16: return max_blocks_dt<DG_C32_F16>(p);
    case DG_C32_BF16: return max_blocks_dt<DG_C32_BF16>(p);
    }
    return 1;
}

int dg_max_warps_per_block() { return dg::kMaxWarps; }
