// Gather arm of the degridding kernel: sparse coverage.
//
// When consecutive visibilities rarely share a footprint (short or sparse
// lists, the regime of the paper's kernels D2 and D4, Section "Results"),
// every visibility reads its own 8 x 8 x 4 footprint, 2 KB in complex64 or
// 1 KB in FP16/BF16, and the sum is bound by how many footprint bytes are
// in flight from L2, not by arithmetic.  The footprint-cache kernel builds
// one footprint at a time per warp, with the loads in registers; here the
// footprints travel by TMA (one tensor copy per footprint: a box of 8 rows of
// the stack, each row the 32 elements of the footprint plus 16 bytes) into
// shared memory, completing on an mbarrier per slot: a warp copies the next
// stage of four footprints while it sums the current one, and the copy of a
// stage costs it one instruction.  The rate is bytes in flight over L2
// latency, and shared memory bounds the bytes: the CTA holds as many warps
// as their two slots each fit (12 for complex64, 22 for FP16/BF16), which
// measured faster than fewer warps with three or four slots each.  (One bulk
// copy per 256-byte row ran slower: the copy engine's per-request cost, not
// bytes, bounded it.)
//
// A warp walks chunks in batches of 32 visibilities (lane i snaps visibility
// i of the batch, as in the other kernels) and each batch in stages of four:
//   issue:   lane v starts the tensor copy of visibility v of stage n + 1,
//            sixteen lanes copy the g_u and g_v rows (cp.async);
//   sum:     stage n, lane 8v + b: row b of visibility v,
//            R_b = sum_a g_u[a] sum_c g_w[c] s[b][a][c];
//   reduce:  within the 8 lanes of a visibility, pairing rows (2j, 2j + 1)
//            with g_v and adding the pair sums as (j, j ^ 2), then (j, j ^ 1).
// Every operation and its order match the footprint-cache kernel (M entries
// as FMA chains over c, then the a sum, then the quarter and pair sums), so
// the two arms agree bit for bit; the compensated form mirrors its TwoSum
// reduction.  The box is 16 bytes wider than a footprint row, so row b lands
// 16 b bytes past a 128-byte boundary and the 8 rows that the 8 lanes of a
// visibility read at once sit in 8 different bank groups (the extra 16 bytes
// are the next column's first samples, or zeros past the edge of the stack).
//
// Waits on the mbarriers are bounded: a wait that gives up records
// kFlagTimeout in the plan's status, waits (bounded again) for the warp's
// copies still in flight and ends the warp.
//
// Requirements (checked by the host): nz = 4, a separable G_uv table, a
// 16-byte aligned subgrid stack.
#include "pipeline.cuh"
#include "tma.cuh"

namespace dg {
namespace {

#ifndef DG_GATHER_STAGES
#define DG_GATHER_STAGES 2          // slots per warp: stages in flight while one is summed, plus one
#endif
#ifndef DG_GATHER_WARPS_C64
#define DG_GATHER_WARPS_C64 12      // warps per CTA (one CTA per SM), complex64 storage
#endif
#ifndef DG_GATHER_WARPS_16
#define DG_GATHER_WARPS_16 22       // warps per CTA, FP16 / BF16 storage
#endif

constexpr int kGVis = 4;            // visibilities per stage (8 lanes each)
constexpr int kGStages = DG_GATHER_STAGES;

// Polls of a warp's wait for a stage before it sums it.  The product build
// waits up to kSpinLimit polls for every stage.  The library variant that
// tests the timeout path waits normally for a warp's first
// DG_GATHER_SUM_WAIT_FROM stages and then with a limit of
// DG_GATHER_SUM_WAIT_POLLS (0: the wait gives up at once, while the stage's
// copies are in flight), so every warp that gets that far records the
// timeout and stops.  The wait for the copies still in flight after a
// timeout always keeps the full bound, so every copy a warp issued has
// landed before the warp ends.
#ifndef DG_GATHER_SUM_WAIT_POLLS
#define DG_GATHER_SUM_WAIT_POLLS kSpinLimit
#endif
#ifndef DG_GATHER_SUM_WAIT_FROM
#define DG_GATHER_SUM_WAIT_FROM 0
#endif
constexpr int kSumWaitPolls = DG_GATHER_SUM_WAIT_POLLS;
constexpr int kSumWaitFrom = DG_GATHER_SUM_WAIT_FROM;

template <int DT>
struct GatherShape {
    static constexpr int kPitch = FootprintBox<DT>::kPitch;              // box row in shared memory
    static constexpr int kWarps = DT == DG_C64 ? DG_GATHER_WARPS_C64 : DG_GATHER_WARPS_16;
};

template <int DT>
struct alignas(128) GatherSlot {
    unsigned char data[kGVis][kUV][GatherShape<DT>::kPitch];   // [v][row b][bytes of the row]
    float4 rows[kGVis][2][2];                                   // [v][g_u, g_v][half]
    unsigned long long bar;                                     // mbarrier: the stage's copies
    int key[kGVis];                                             // footprint start, -1 = invalid
    int fw[kGVis];                                              // w-kernel row
    long long out0;                                             // output index of visibility 0
    int n;                                                      // visibilities in the stage (1..4)
    int s;                                                      // subgrid
};

// Issue side of a warp: the batch being copied and the next one.
struct GatherIssue {
    Batch b;            // batch whose stages are being issued (n = 0: none left)
    int q;              // next stage of b
    int key, fw, fu, fv;
    int xe, y0;         // footprint start: element in its row, row in the subgrid
    Batch nb;           // the batch after b, its coordinates in registers
    Coords3 nc;
};

__device__ __forceinline__ void snap_batch(GatherIssue &is, const Coords3 &c, const Geometry &g,
                                           DeviceStatus *status, int lane)
{
    const bool in = lane < is.b.n;
    VisCoords vc;
    bool valid = in && visibility_coords(c.u, c.v, c.w, g, vc);
#ifdef DEGRID_BOUNDS_CHECK
    if (valid)
        valid = indices_in_bounds((vc.y0 * g.nx + vc.x0) * g.nz + vc.z0, vc.fu, vc.fv, vc.fw, g, status);
#endif
    is.key = valid ? (vc.y0 * g.nx + vc.x0) * g.nz + vc.z0 : -1;
    is.fw = valid ? vc.fw : 0;
    is.fu = valid ? vc.fu : 0;
    is.fv = valid ? vc.fv : 0;
    is.xe = valid ? vc.x0 * g.nz + vc.z0 : 0;
    is.y0 = valid ? vc.y0 : 0;
    const unsigned bad = __ballot_sync(kFull, in && !valid);
    if (lane == 0 && bad)
        atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
}

// Issues the copies of the next stage into `sl` (its mbarrier's phase
// completes when they have landed); returns whether a stage was issued.
template <int DT>
__device__ __forceinline__ int issue_stage(GatherIssue &is, GatherSlot<DT> &sl, ClaimerT<kBatch> &cl,
                                           const CUtensorMap *map, const float *__restrict__ guv,
                                           const double *__restrict__ uvw, const Geometry &g,
                                           DeviceStatus *status, int lane)
{
    if (is.b.n == 0) {
        cp_async_commit();
        return 0;
    }
    const int first = kGVis * is.q;
    const int n = min(kGVis, is.b.n - first);
    const uint32_t bar = smem_u32(&sl.bar);
    {   // footprints: lane v < 4, one tensor copy each
        const int v = lane & 3;
        const int kv = __shfl_sync(kFull, is.key, first + v);
        const int xe = __shfl_sync(kFull, is.xe, first + v);
        const int y0 = __shfl_sync(kFull, is.y0, first + v);
        const bool copy = lane < kGVis && v < n && kv >= 0;
        const int nvalid = __popc(__ballot_sync(kFull, copy));
        // the slot's earlier contents were read through the generic proxy;
        // the tensor copies write it through the async proxy
        fence_proxy_async();
        if (lane == 0)
            mbar_arrive_expect_tx(bar, (unsigned)nvalid * (unsigned)sizeof(sl.data[0]));
        __syncwarp();
        if (copy)
            tensor_copy_2d(smem_u32(&sl.data[v][0][0]), map, xe, is.b.s * g.ny + y0, bar);
        const int fwv = __shfl_sync(kFull, is.fw, first + v);
        if (lane < kGVis) {                             // metadata, read back by the summing lanes
            sl.key[lane] = v < n ? kv : -1;
            sl.fw[lane] = fwv;
        }
        if (lane == 0) {
            sl.out0 = is.b.b0 + first;
            sl.n = n;
            sl.s = is.b.s;
        }
    }
    {   // g_u and g_v rows: lane 4v + 2 which + half, lanes 0..15
        const int v = (lane >> 2) & 3, which = (lane >> 1) & 1, half = lane & 1;
        const int kv = __shfl_sync(kFull, is.key, first + v);
        const int fu = __shfl_sync(kFull, is.fu, first + v);
        const int fv = __shfl_sync(kFull, is.fv, first + v);
        if (lane < 16 && v < n && kv >= 0)
            cp_async16(smem_u32(&sl.rows[v][which][half]), guv + (size_t)(which ? fv : fu) * kUVRow + 4 * half);
        cp_async_commit();
    }
    if (++is.q * kGVis >= is.b.n) {                     // batch done: snap the next one
        is.b = is.nb;
        is.q = 0;
        if (is.b.n > 0) {
            snap_batch(is, is.nc, g, status, lane);
            is.nb = cl.advance(is.b);
            is.nc = load_uvw(uvw, is.nb, lane);
        }
    }
    return 1;
}

// The four elements (z = 0..3) of footprint column a of row b, as float2.
template <int DT>
__device__ __forceinline__ void column(const GatherSlot<DT> &sl, int v, int b, int a, float2 (&s)[4])
{
    if constexpr (DT == DG_C64) {
        const float4 *r = reinterpret_cast<const float4 *>(&sl.data[v][b][0]);
        const float4 p = r[2 * a], q = r[2 * a + 1];
        s[0] = make_float2(p.x, p.y);
        s[1] = make_float2(p.z, p.w);
        s[2] = make_float2(q.x, q.y);
        s[3] = make_float2(q.z, q.w);
    } else {
        const uint4 p = reinterpret_cast<const uint4 *>(&sl.data[v][b][0])[a];
        s[0] = Storage<DT>::cvt(p.x);
        s[1] = Storage<DT>::cvt(p.y);
        s[2] = Storage<DT>::cvt(p.z);
        s[3] = Storage<DT>::cvt(p.w);
    }
}

__device__ __forceinline__ float two_sum_g(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// Sums the stage in `sl` and stores its visibilities.
template <int DT, bool COMP>
__device__ __forceinline__ void sum_stage(const GatherSlot<DT> &sl, const float4 *wtab,
                                          const float *__restrict__ gwt, const float *__restrict__ scale,
                                          float2 *__restrict__ vis_out, int lane)
{
    const int v = lane >> 3, b = lane & 7;
    const int key = sl.key[v];
    const int fw = sl.fw[v];
    const float4 gw = wtab ? wtab[fw] : __ldg(reinterpret_cast<const float4 *>(gwt) + fw);
    const float4 u0 = sl.rows[v][0][0], u1 = sl.rows[v][0][1];
    const float gu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    const float4 vq = sl.rows[v][1][b >> 2];
    const float gv_e = (b & 2) ? vq.z : vq.x;           // g_v[b & ~1]
    const float gv_o = (b & 2) ? vq.w : vq.y;           // g_v[b | 1]
    // R_b = sum_a g_u[a] M[b][a], M[b][a] = sum_c g_w[c] s[b][a][c]: the
    // same FMA chains as the footprint-cache kernel, as (re, im) pairs
    float2 R = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < kUV; ++a) {
        float2 s[4];
        column<DT>(sl, v, b, a, s);
        float2 m = __fmul2_rn(s[0], make_float2(gw.x, gw.x));
        m = __ffma2_rn(s[1], make_float2(gw.y, gw.y), m);
        m = __ffma2_rn(s[2], make_float2(gw.z, gw.z), m);
        m = __ffma2_rn(s[3], make_float2(gw.w, gw.w), m);
        R = a == 0 ? __fmul2_rn(m, make_float2(gu[0], gu[0])) : __ffma2_rn(m, make_float2(gu[a], gu[a]), R);
    }
    // quarter j = b >> 1: g_v[2j + 1] R_{2j + 1} + g_v[2j] R_{2j}
    const float2 Rn = make_float2(__shfl_xor_sync(kFull, R.x, 1), __shfl_xor_sync(kFull, R.y, 1));
    const float2 Re = (b & 1) ? Rn : R, Ro = (b & 1) ? R : Rn;
    const float2 Q = __ffma2_rn(Ro, make_float2(gv_o, gv_o), __fmul2_rn(Re, make_float2(gv_e, gv_e)));
    // (Q_j + Q_{j^2}) + (Q_{j^1} + Q_{j^3})
    float2 V;
    if (COMP) {
        float2 e0, e;
        const float2 S = make_float2(two_sum_g(Q.x, __shfl_xor_sync(kFull, Q.x, 4), e0.x),
                                     two_sum_g(Q.y, __shfl_xor_sync(kFull, Q.y, 4), e0.y));
        V.x = two_sum_g(S.x, __shfl_xor_sync(kFull, S.x, 2), e.x);
        V.y = two_sum_g(S.y, __shfl_xor_sync(kFull, S.y, 2), e.y);
        e.x += e0.x + __shfl_xor_sync(kFull, e0.x, 2);
        e.y += e0.y + __shfl_xor_sync(kFull, e0.y, 2);
        V.x += e.x;
        V.y += e.y;
    } else {
        const float2 S = make_float2(Q.x + __shfl_xor_sync(kFull, Q.x, 4), Q.y + __shfl_xor_sync(kFull, Q.y, 4));
        V = make_float2(S.x + __shfl_xor_sync(kFull, S.x, 2), S.y + __shfl_xor_sync(kFull, S.y, 2));
    }
    if (DT != DG_C64) {
        const float sc = __ldg(scale + sl.s);
        V = __fmul2_rn(V, make_float2(sc, sc));
    }
    if (b == 0 && v < sl.n)
        vis_out[sl.out0 + v] = key >= 0 ? V : make_float2(0.f, 0.f);
}

template <int DT, bool COMP>
__global__ void __launch_bounds__(GatherShape<DT>::kWarps * kWarp, 1)
degrid_gather_kernel(const Geometry g, const __grid_constant__ CUtensorMap tmap,
                     const float *__restrict__ scale, const double *__restrict__ uvw,
                     const float *__restrict__ guv, const float *__restrict__ gwt, const Schedule sched,
                     float2 *__restrict__ vis_out, DeviceStatus *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GatherSlot<DT> *slots = reinterpret_cast<GatherSlot<DT> *>(smem_raw + wtable_bytes(g)) +
                            (threadIdx.x >> 5) * kGStages;
    const float4 *wtab = load_wtable(g, gwt, smem_raw);
    const int lane = threadIdx.x & 31;

    pdl_wait();                         // the chunk table is complete
    ClaimerT<kBatch> cl(sched, lane, Prefetch{uvw, 3 * (int)sizeof(double), nullptr, 0});
    GatherIssue is;
    is.q = 0;
    is.b = cl.claim();
    is.key = -1;
    is.fw = is.fu = is.fv = 0;
    is.nb = Batch{0, 0, 0, 0};
    is.nc = Coords3{0.0, 0.0, 0.0};
    if (is.b.n > 0) {
        snap_batch(is, load_uvw(uvw, is.b, lane), g, status, lane);
        is.nb = cl.advance(is.b);
        is.nc = load_uvw(uvw, is.nb, lane);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kGStages; ++k)
            mbar_init(smem_u32(&slots[k].bar), 1);
        fence_mbarrier_init();
    }
    __syncwarp();
    int issued = 0;
#pragma unroll
    for (int k = 0; k < kGStages - 1; ++k)
        issued += issue_stage<DT>(is, slots[k], cl, &tmap, guv, uvw, g, status, lane);
    int done = 0;
    for (; done < issued; ++done) {
        // the slot summed in the previous iteration takes stage done + kGStages - 1
        issued += issue_stage<DT>(is, slots[(done + kGStages - 1) % kGStages], cl, &tmap, guv, uvw, g,
                                  status, lane);
        GatherSlot<DT> &sl = slots[done % kGStages];
        cp_async_wait<kGStages - 1>();                  // this lane's row copies of stage `done`
        if (!mbar_wait_bounded(smem_u32(&sl.bar), (unsigned)(done / kGStages) & 1u,
                               done < kSumWaitFrom ? kSpinLimit : kSumWaitPolls)) {
            if (lane == 0)
                atomicOr(&status->flags, kFlagTimeout);
            break;
        }
        __syncwarp();                                   // every lane's row copies
        sum_stage<DT, COMP>(sl, wtab, gwt, scale, vis_out, lane);
        __syncwarp();
    }
    // after a timeout: wait (bounded, the full kSpinLimit) for the copies
    // still in flight
    for (; done < issued; ++done)
        mbar_wait_bounded(smem_u32(&slots[done % kGStages].bar), (unsigned)(done / kGStages) & 1u, kSpinLimit);
    cp_async_wait<0>();
}

size_t gather_smem(const degrid_plan *p, int warps, size_t slot_bytes)
{
    return wtable_bytes_host(p->geo) + slot_bytes * kGStages * (size_t)warps;
}

template <int DT, bool COMP>
cudaError_t launch_gather(degrid_plan *p, cudaStream_t st, const void *subgrids, int n_subgrids,
                          const float *scale, const double *uvw, float2 *out, const Schedule &sched,
                          int grid_blocks)
{
    constexpr int kWarps = GatherShape<DT>::kWarps;
    const size_t smem = gather_smem(p, kWarps, sizeof(GatherSlot<DT>));
    static std::atomic<size_t> smem_table[kMaxDevices];
    cudaError_t e = dg_open_smem(dg_smem_record(smem_table, p->device), degrid_gather_kernel<DT, COMP>, smem);
    if (e != cudaSuccess)
        return e;
    CUtensorMap map;
    e = encode_footprint_map<DT>(p, subgrids, n_subgrids, &map);
    if (e != cudaSuccess)
        return e;
    return launch_pdl(degrid_gather_kernel<DT, COMP>, dim3(grid_blocks), dim3(kWarps * kWarp), smem, st,
                      p->geo, map, scale, uvw, (const float *)p->guv, (const float *)p->gw, sched, out,
                      p->status);
}

template <int DT>
cudaError_t launch_gather_dt(degrid_plan *p, cudaStream_t st, const void *subgrids, int n_subgrids,
                             const float *scale, const double *uvw, float2 *out, const Schedule &sched,
                             int grid_blocks)
{
    return p->compensated
               ? launch_gather<DT, true>(p, st, subgrids, n_subgrids, scale, uvw, out, sched, grid_blocks)
               : launch_gather<DT, false>(p, st, subgrids, n_subgrids, scale, uvw, out, sched, grid_blocks);
}

}  // namespace
}  // namespace dg

int dg_gather_warps(dg_dtype dtype)
{
    using namespace dg;
    return dtype == DG_C64 ? GatherShape<DG_C64>::kWarps : GatherShape<DG_C32_F16>::kWarps;
}

bool dg_gather_supported(const degrid_plan *p)
{
    return p->geo.nz == dg::kW && p->guv2 == nullptr;
}

cudaError_t dg_launch_gather(degrid_plan *p, cudaStream_t st, const void *subgrids, int n_subgrids,
                             const float *scale, const double *uvw, float *out_f, int grid_blocks)
{
    using namespace dg;
    Schedule sched{p->chunks, p->n_chunks, p->work_counter};
    float2 *out = reinterpret_cast<float2 *>(out_f);
    switch (p->dtype) {
    case DG_C64:
        return launch_gather_dt<DG_C64>(p, st, subgrids, n_subgrids, scale, uvw, out, sched, grid_blocks);
    case DG_C32_F16:
        return launch_gather_dt<DG_C32_F16>(p, st, subgrids, n_subgrids, scale, uvw, out, sched, grid_blocks);
    case DG_C32_BF16:
        return launch_gather_dt<DG_C32_BF16>(p, st, subgrids, n_subgrids, scale, uvw, out, sched, grid_blocks);
    }
    return cudaErrorInvalidValue;
}
