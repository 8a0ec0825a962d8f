// Degridding kernel (paper Section "Implementation": kernel D1 and its
// variants), re-designed for sm_103a.
//
// Work decomposition.  A persistent grid of warps claims chunks of
// consecutive visibilities of one subgrid (schedule.cu) and walks each chunk
// in batches of 32 visibilities.  Claims are pipelined: a warp holds the
// descriptor of its next chunk while working on the current one.
//
// Per batch, three stages overlap across consecutive batches of a warp:
//  1. the FP64 coordinates of batch n + 2 are loaded into registers;
//  2. for batch n + 1, lane i snaps visibility i (exact integer rint of the
//     coordinates, internal.cuh) and the warp fetches the three GCF rows of
//     every visibility with TMA tile::gather4 copies (4 table rows per copy)
//     into the warp's shared-memory stage, completion tracked by an mbarrier;
//  3. batch n is summed from the stage that arrived.
// The paper's D1 computes the coordinates of its N_b visibilities
// cooperatively into shared memory first; here that step is both overlapped
// with the sums and taken off the load/store pipe by the TMA engine.
//
// Footprint sum.  Each quarter-warp (8 lanes) computes one visibility; the
// warp does 4 visibilities per step, 8 steps per batch.  Lane (a-pair, c-pair)
// holds the 4 footprint columns (a0 + i, c0 + j), i, j in {0, 1}, of all 8
// rows b in registers (32 complex values) and reloads them only when the
// footprint start changes: consecutive visibilities of a dense list share the
// footprint (the reuse the paper notes for D1), so the subgrid is read once
// per footprint.  Each lane accumulates along v (b) as in D1, with one packed
// FP32 FMA (FFMA2) per complex x real product; the GCF tables are stored with
// every tap duplicated, so a 16-byte shared load yields two ready (g, g)
// operand pairs.  The four column sums are then weighted by g_u and g_w.
// A batch whose 32 visibilities share one valid footprint takes a branch-free
// path; otherwise every quarter checks and reloads its own footprint.
//
// Reduction and output.  The 8 partials of a quarter are reduced with a
// transposing butterfly (3 shuffle levels that halve the live values), after
// which every lane holds one whole visibility; the warp writes its 32
// results into one contiguous 256-byte segment (the paper's bulk
// contiguous write-out, without the shared-memory staging).
#include "internal.cuh"

namespace dg {
namespace {

#ifndef DG_STAGING_TMA
#define DG_STAGING_TMA 0     // GCF rows staged by TMA tile::gather4 (1) or cp.async (0)
#endif

#ifndef DG_DEGRID_MAX_WARPS
#define DG_DEGRID_MAX_WARPS 8
#endif
#ifndef DG_PINNED_UVW_LOADS
#define DG_PINNED_UVW_LOADS 1
#endif
#ifndef DG_FOOTPRINT_ASM_LOADS
#define DG_FOOTPRINT_ASM_LOADS 1   // footprint loads the compiler may not re-issue
#endif

constexpr int kMaxWarps = DG_DEGRID_MAX_WARPS;   // per CTA
constexpr int kBatch = 32;                  // visibilities per warp batch
constexpr int kUVRow = 16;                  // floats per duplicated uv row (64 B)
constexpr int kWRow = 8;                    // floats per duplicated w row (32 B)
constexpr unsigned kStageBytes = kBatch * 2 * kUVRow * 4;  // TMA bytes per batch: g_u + g_v rows
// The duplicated w table (O_w rows of 32 B) is kept in every CTA's shared
// memory when it is at most this large (O_w <= 512); otherwise its rows are
// fetched per batch like the uv rows.  Along a dense list f_w stays constant
// for thousands of visibilities, so per-batch w fetches would make every warp
// on the GPU hit the same few L2 lines.
constexpr int kMaxWTableBytes = 16 * 1024;

struct alignas(128) Stage {
    float gu[kBatch][kUVRow];   // TMA destination: g_uv[fu] duplicated
    float gv[kBatch][kUVRow];   // TMA destination: g_uv[fv] duplicated
    float gw[kBatch][kWRow];    // TMA destination: g_w[fw] duplicated
    int key[kBatch];            // footprint start (y0 * nx + x0) * nz + z0, -1 invalid
    int meta;                   // common key if all 32 share one valid footprint, else -1
};

struct alignas(128) WarpSmem {
    Stage st[2];
    float2 slow[8][kWarp];      // per-step partials on the mixed-footprint path
    unsigned long long bar[2];  // one mbarrier per stage
};

// ---- PTX wrappers ---------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

// Four rows (r0..r3) of a 2D tensor, column 0, into consecutive shared
// memory rows; completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap *tm, int r0, int r1,
                                            int r2, int r3, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
        : "memory");
}

// 16-byte asynchronous global -> shared copy (L2 only), grouped per batch.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }

// ---- footprint registers ----------------------------------------------------

// One footprint sample as (re, im).  The loads are volatile inline PTX so
// that, under register pressure, the compiler keeps (or spills) the values
// instead of re-issuing read-only global loads inside the hot loop.
template <int DT>
__device__ __forceinline__ float2 load_sample(const void *sub, int64_t i)
{
#if DG_FOOTPRINT_ASM_LOADS
    if (DT == DG_C64) {
        float2 v;
        asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];"
                     : "=f"(v.x), "=f"(v.y)
                     : "l"(reinterpret_cast<const float2 *>(sub) + i));
        return v;
    } else {
        unsigned u;
        asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(u) : "l"(reinterpret_cast<const unsigned *>(sub) + i));
        if (DT == DG_C32_F16) {
            __half2 h = *reinterpret_cast<const __half2 *>(&u);
            return __half22float2(h);
        }
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
#else
    return Storage<DT>::load(sub, i);
#endif
}

// B[k][e][i][j] = s[y0 + b][x0 + a0 + i][z0 + c0 + j] with b = 2 * ((k + quarter) & 3) + e.
// The row order is rotated by quarter so that, at every shared-memory load of
// a step, the four quarters read different 16-byte chunks of their g_v rows
// (no bank conflicts), while the register slots stay compile-time indices.
template <int DT>
__device__ __forceinline__ void load_footprint(float2 (&B)[4][2][2][2], const void *sub,
                                               int64_t base, int key, int quarter, int a0, int c0,
                                               const Geometry &g)
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j4 = (k + quarter) & 3;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t row = base + key + (int64_t)(2 * j4 + e) * g.row_stride;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    B[k][e][i][j] = load_sample<DT>(sub, row + (a0 + i) * g.nz + (c0 + j));
        }
    }
}

// Partial sum of visibility r of the stage over this lane's 4 columns:
// sum_b g_v[b] * (g_u[a0] g_w[c0] B(a0,c0) + ...), 38 packed FP32 operations.
__device__ __forceinline__ float2 footprint_step(const float2 (&B)[4][2][2][2], const Stage &S,
                                                 int r, int quarter, int ap, int cp)
{
    const float4 *gvrow = reinterpret_cast<const float4 *>(S.gv[r]);
    float2 acc[2][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 gk = gvrow[(k + quarter) & 3];
        const float2 g0 = lo2(gk), g1 = hi2(gk);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                acc[i][j] = k == 0 ? __fmul2_rn(B[0][0][i][j], g0)
                                   : __ffma2_rn(B[k][0][i][j], g0, acc[i][j]);
                acc[i][j] = __ffma2_rn(B[k][1][i][j], g1, acc[i][j]);
            }
    }
    const float4 gu4 = reinterpret_cast<const float4 *>(S.gu[r])[ap];
    const float4 gw4 = reinterpret_cast<const float4 *>(S.gw[r])[cp];
    float2 t0 = __fmul2_rn(acc[0][0], lo2(gu4));
    t0 = __ffma2_rn(acc[1][0], hi2(gu4), t0);
    float2 t1 = __fmul2_rn(acc[0][1], lo2(gu4));
    t1 = __ffma2_rn(acc[1][1], hi2(gu4), t1);
    float2 p = __fmul2_rn(t0, lo2(gw4));
    return __ffma2_rn(t1, hi2(gw4), p);
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

// ---- batch stream ---------------------------------------------------------

struct Batch {
    int s;          // subgrid
    int n;          // visibilities in this batch (1..32), 0 = none
    long long b0;   // first visibility
    long long end;  // end of the chunk
};

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

__device__ __forceinline__ void load_uvw(const double *__restrict__ uvw, const Batch &b, int lane,
                                         double &u, double &v, double &w)
{
    if (lane < b.n) {
        const double *p = uvw + 3 * (b.b0 + lane);
#if DG_PINNED_UVW_LOADS
        // volatile: the loads stay where they are issued (two batches ahead of
        // their use) instead of being sunk to the use under register pressure
        asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(u) : "l"(p));
        asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p + 1));
        asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(w) : "l"(p + 2));
#else
        u = __ldg(p);
        v = __ldg(p + 1);
        w = __ldg(p + 2);
#endif
    } else {
        u = v = w = 0.0;
    }
}

// Stage 2 for one batch: coordinates, keys, and the copies of the three
// duplicated GCF rows of every visibility into the stage.
__device__ __forceinline__ void issue_batch(const Batch &b, double u, double v, double w,
                                            const Geometry &g, Stage &S, uint32_t bar,
                                            const CUtensorMap *tm_uv, const CUtensorMap *tm_w,
                                            const float *__restrict__ guv2,
                                            const float *__restrict__ gw2, const float4 *wtab,
                                            int lane, DeviceStatus *status)
{
    const bool in = lane < b.n;
    VisCoords vc;
    const bool valid = in && visibility_coords(u, v, w, g, vc);
    const int key = valid ? (vc.y0 * g.nx + vc.x0) * g.nz + vc.z0 : -1;
    const int fu = valid ? vc.fu : 0, fv = valid ? vc.fv : 0, fw = valid ? vc.fw : 0;
    S.key[lane] = key;
    const int key0 = __shfl_sync(kFull, key, 0);
    const bool uniform = __all_sync(kFull, key == key0) && key0 >= 0;
    if (lane == 0)
        S.meta = uniform ? key0 : -1;
    const unsigned bad = __ballot_sync(kFull, in && !valid);
    if (lane == 0 && bad)
        atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
    // g_w rows: from the CTA's copy of the table when there is one
    if (wtab) {
        float4 *dst = reinterpret_cast<float4 *>(S.gw[lane]);
        dst[0] = wtab[2 * fw];
        dst[1] = wtab[2 * fw + 1];
    }
#if DG_STAGING_TMA
    (void)guv2;
    (void)tm_w;
    // lanes 0-7 gather g_u rows, 8-15 g_v rows, 4 rows per lane
    const int grp = lane >> 3, jj = lane & 7;
    int r[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int src = 4 * jj + m;
        const int xu = __shfl_sync(kFull, fu, src);
        const int xv = __shfl_sync(kFull, fv, src);
        r[m] = grp == 0 ? xu : xv;
    }
    fence_proxy_async();
    __syncwarp();
    if (lane == 0)
        mbar_arrive_expect_tx(bar, kStageBytes);
    __syncwarp();
    if (grp < 2)
        tma_gather4(grp == 0 ? smem_u32(S.gu[4 * jj]) : smem_u32(S.gv[4 * jj]), tm_uv, r[0], r[1],
                    r[2], r[3], bar);
    if (!wtab) {
        const int cw = lane & 1;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int rr = (lane >> 1) + 16 * m;
            const int xw = __shfl_sync(kFull, fw, rr);
            cp_async16(smem_u32(&S.gw[rr][4 * cw]), gw2 + (size_t)xw * kWRow + 4 * cw);
        }
        cp_async_commit();
    }
#else
    (void)bar;
    (void)tm_uv;
    (void)tm_w;
    // 4 lanes per 64-byte uv row (one 16-byte chunk each), 2 per 32-byte w row
    const int cu = lane & 3, cw = lane & 1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int r = (lane >> 2) + 8 * m;
        const int xu = __shfl_sync(kFull, fu, r);
        const int xv = __shfl_sync(kFull, fv, r);
        cp_async16(smem_u32(&S.gu[r][4 * cu]), guv2 + (size_t)xu * kUVRow + 4 * cu);
        cp_async16(smem_u32(&S.gv[r][4 * cu]), guv2 + (size_t)xv * kUVRow + 4 * cu);
    }
    if (!wtab) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            const int r = (lane >> 1) + 16 * m;
            const int xw = __shfl_sync(kFull, fw, r);
            cp_async16(smem_u32(&S.gw[r][4 * cw]), gw2 + (size_t)xw * kWRow + 4 * cw);
        }
    }
    cp_async_commit();
#endif
}

#ifndef DG_DEGRID_MIN_BLOCKS
#define DG_DEGRID_MIN_BLOCKS 2   // resident CTAs per SM the register budget is sized for
#endif

template <int DT>
__global__ void __launch_bounds__(kMaxWarps * kWarp, DG_DEGRID_MIN_BLOCKS)
degrid_kernel(const Geometry g, const void *__restrict__ subgrids, const float *__restrict__ scale,
              const double *__restrict__ uvw, const __grid_constant__ CUtensorMap tm_uv,
              const __grid_constant__ CUtensorMap tm_w, const float *__restrict__ guv2,
              const float *__restrict__ gw2, const Schedule sched,
              float2 *__restrict__ vis_out, DeviceStatus *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // [w table (optional)] [one WarpSmem per warp]
    const int wtab_bytes = g.w_table_rows > 0 ? ((g.w_table_rows * kWRow * 4 + 127) & ~127) : 0;
    WarpSmem &ws = reinterpret_cast<WarpSmem *>(smem_raw + wtab_bytes)[threadIdx.x >> 5];
    const float4 *wtab = nullptr;
    if (wtab_bytes) {
        float4 *t = reinterpret_cast<float4 *>(smem_raw);
        const float4 *src = reinterpret_cast<const float4 *>(gw2);
        for (int i = threadIdx.x; i < g.w_table_rows * (kWRow / 4); i += blockDim.x)
            t[i] = __ldg(src + i);
        __syncthreads();
        wtab = t;
    }
    const int lane = threadIdx.x & 31;
    const int quarter = lane >> 3, q = lane & 7, ap = q >> 1, cp = q & 1;
    const int a0 = 2 * ap, c0 = 2 * cp;
    const uint32_t bar0 = smem_u32(&ws.bar[0]), bar1 = smem_u32(&ws.bar[1]);
    if (lane == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        fence_barrier_init();
    }
    __syncwarp();

    Claimer claimer(sched, lane);
    Batch bB = claimer.claim();         // tables in flight
    if (bB.n == 0)
        return;
    double u, v, w;
    load_uvw(uvw, bB, lane, u, v, w);
    issue_batch(bB, u, v, w, g, ws.st[0], bar0, &tm_uv, &tm_w, guv2, gw2, wtab, lane, status);
    Batch bC = claimer.advance(bB);     // coordinates in registers
    load_uvw(uvw, bC, lane, u, v, w);

    uint32_t parity = 0;                // bit s: parity of the next phase of stage s
    int stage = 0;
    int cur = -2, cur_s = -1;           // footprint held in B (key, subgrid)
    float2 B[4][2][2][2];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    B[k][e][i][j] = make_float2(0.f, 0.f);

    while (bB.n > 0) {
        const Batch bA = bB;            // computed in this iteration
        const int sA = stage;
        bB = bC;
        if (bB.n > 0)
            issue_batch(bB, u, v, w, g, ws.st[sA ^ 1], sA ? bar0 : bar1, &tm_uv, &tm_w, guv2, gw2,
                        wtab, lane, status);
        bC = claimer.advance(bC);
        load_uvw(uvw, bC, lane, u, v, w);

#if DG_STAGING_TMA
        if (!mbar_wait(sA ? bar1 : bar0, (parity >> sA) & 1)) {
            if (lane == 0)
                atomicOr(&status->flags, kFlagTimeout);
            if (bB.n > 0)       // let the copies already issued land before leaving
                mbar_wait(sA ? bar0 : bar1, (parity >> (sA ^ 1)) & 1);
            return;
        }
        parity ^= 1u << sA;
        if (!wtab) {
            if (bB.n > 0)
                cp_async_wait<1>();
            else
                cp_async_wait<0>();
        }
        __syncwarp();
#else
        if (bB.n > 0)
            cp_async_wait<1>();     // the stage of batch A; batch B may stay in flight
        else
            cp_async_wait<0>();
        __syncwarp();
#endif

        const Stage &S = ws.st[sA];
        if (bA.s != cur_s) {
            cur_s = bA.s;
            cur = -2;
        }
        const int64_t base = (int64_t)bA.s * g.plane;
        float2 P[8];
        const int meta = S.meta;
        if (meta >= 0) {
            if (meta != cur) {
                load_footprint<DT>(B, subgrids, base, meta, quarter, a0, c0, g);
                cur = meta;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
                P[t] = footprint_step(B, S, 4 * t + quarter, quarter, ap, cp);
        } else {
#pragma unroll 1
            for (int t = 0; t < 8; ++t) {
                const int r = 4 * t + quarter;
                const int kv = S.key[r];
                if (kv != cur) {
                    cur = kv;
                    if (kv >= 0)
                        load_footprint<DT>(B, subgrids, base, kv, quarter, a0, c0, g);
                }
                ws.slow[t][lane] = kv >= 0 ? footprint_step(B, S, r, quarter, ap, cp)
                                           : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int t = 0; t < 8; ++t)
                P[t] = ws.slow[t][lane];
        }
        float2 V = quarter_reduce(P, q);
        const int r_out = 4 * q + quarter;
        if (DT != DG_C64)
            V = __fmul2_rn(V, make_float2(__ldg(scale + bA.s), __ldg(scale + bA.s)));
        if (r_out < bA.n)
            vis_out[bA.b0 + r_out] = V;
        __syncwarp();
        stage ^= 1;
    }
}

size_t smem_bytes(const degrid_plan *p, int warps)
{
    const size_t wt = p->geo.w_table_rows > 0 ? ((size_t)p->geo.w_table_rows * kWRow * 4 + 127) & ~(size_t)127 : 0;
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
    degrid_kernel<DT><<<grid_blocks, threads, smem, st>>>(p->geo, subgrids, scale, uvw, p->tm_uv2,
                                                           p->tm_w2, p->guv2, p->gw2, sched, out,
                                                           p->status);
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
