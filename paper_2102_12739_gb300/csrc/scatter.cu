// Gridding (the adjoint) for scattered coverage.
//
// The adjoint kernel (adjoint.cu) accumulates the scatter of a run of
// visibilities that share a footprint in registers and adds it to the
// subgrid with 128 16-byte vector reductions (256 float2 atomics on other
// layouts) when the run ends.  When consecutive visibilities rarely share a
// footprint (sparse or short lists, the regime of the paper's D2/D4
// variants, Section "Results") every visibility is a run of its own and the
// atomics bound it.  This kernel writes each
// visibility's whole contribution,
//   tile[b][a][c] = g_w[c] (g_u[a] (y g_v[b]))    (the adjoint kernel's rounding),
// into shared memory in the layout of the stack (8 rows of 32 samples) and
// hands it to the copy engine as one tensor reduce-add
// (cp.reduce.async.bulk.tensor ... .add), which adds the 2 KB box into the
// subgrid in L2.
//
// A warp walks chunks in batches of 32 visibilities (lane i snaps
// visibility i and loads its value) and each batch in stages of four:
//   issue:  the g_u / g_v rows of stage n + 1 by cp.async, and its metadata;
//   tile:   stage n, lane 8v + a writes column a (all 8 rows, 4 samples) of
//           visibility v's tile;
//   reduce: lane 8v starts the reduce of tile v.
// Each warp has two slots, so a tile is rewritten two stages after its
// reduce started; before that the issuing lane waits until the copy engine
// has read it (cp.async.bulk.wait_group.read, a wait the hardware bounds).
// Invalid visibilities add nothing and are counted.
//
// Requirements (checked by the host): nz = 4 (a footprint row is one
// contiguous piece of the stack), a separable G_uv table, a 16-byte aligned
// output stack.
#include "pipeline.cuh"
#include "tma.cuh"

namespace dg {
namespace {

constexpr int kSVis = 4;            // visibilities per stage (8 lanes each)
constexpr int kSWarps = 12;         // warps per CTA (one CTA per SM)

struct alignas(128) ScatterSlot {
    float tile[kSVis][kUV][kUV * kW * 2];   // [v][row b][2 (4 a + c) + re/im]: the box of the reduce
    float4 rows[kSVis][2][2];               // [v][g_u, g_v][half]
    float2 y[kSVis];                        // visibility values
    int key[kSVis];                         // footprint start, -1: nothing to add
    int fw[kSVis];                          // w-kernel row
    int bx[kSVis], by[kSVis];               // box coordinates: float in the row, row of the stack
    int n;                                  // visibilities in the stage (1..4)
};

// Issue side of a warp: the batch being prepared and the next one.
struct ScatterIssue {
    Batch b;
    int q;                                  // next stage of b
    int key, fw, fu, fv, bx, by;            // this lane's visibility of the batch
    float2 y;
    Batch nb;                               // the batch after b: coordinates and values in registers
    Coords3 nc;
    float2 ny;
};

__device__ __forceinline__ float2 load_vis(const float2 *__restrict__ vis, const Batch &b, int lane)
{
    return lane < b.n ? __ldg(vis + b.b0 + lane) : make_float2(0.f, 0.f);
}

__device__ __forceinline__ void snap_scatter(ScatterIssue &is, const Coords3 &c, const Geometry &g,
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
    is.bx = valid ? 2 * (vc.x0 * g.nz + vc.z0) : 0;
    is.by = valid ? is.b.s * g.ny + vc.y0 : 0;
    const unsigned bad = __ballot_sync(kFull, in && !valid);
    if (lane == 0 && bad)
        atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
}

// Copies the rows and metadata of the next stage into `sl` (one cp.async
// group, empty when no work is left); returns whether a stage was issued.
__device__ __forceinline__ int issue_scatter(ScatterIssue &is, ScatterSlot &sl, ClaimerT<kBatch> &cl,
                                             const float *__restrict__ guv, const double *__restrict__ uvw,
                                             const float2 *__restrict__ vis, const Geometry &g,
                                             DeviceStatus *status, int lane)
{
    if (is.b.n == 0) {
        cp_async_commit();
        return 0;
    }
    const int first = kSVis * is.q;
    const int n = min(kSVis, is.b.n - first);
    {   // g_u and g_v rows: lane 4v + 2 which + half, lanes 0..15
        const int v = (lane >> 2) & 3, which = (lane >> 1) & 1, half = lane & 1;
        const int kv = __shfl_sync(kFull, is.key, first + v);
        const int fu = __shfl_sync(kFull, is.fu, first + v);
        const int fv = __shfl_sync(kFull, is.fv, first + v);
        if (lane < 16 && v < n && kv >= 0)
            cp_async16(smem_u32(&sl.rows[v][which][half]), guv + (size_t)(which ? fv : fu) * kUVRow + 4 * half);
        cp_async_commit();
    }
    {   // metadata
        const int v = lane & 3;
        const int kv = __shfl_sync(kFull, is.key, first + v);
        const int fwv = __shfl_sync(kFull, is.fw, first + v);
        const int bx = __shfl_sync(kFull, is.bx, first + v);
        const int by = __shfl_sync(kFull, is.by, first + v);
        const float yx = __shfl_sync(kFull, is.y.x, first + v);
        const float yy = __shfl_sync(kFull, is.y.y, first + v);
        if (lane < kSVis) {
            sl.key[lane] = v < n ? kv : -1;
            sl.fw[lane] = fwv;
            sl.bx[lane] = bx;
            sl.by[lane] = by;
            sl.y[lane] = make_float2(yx, yy);
        }
        if (lane == 0)
            sl.n = n;
    }
    if (++is.q * kSVis >= is.b.n) {          // batch done: snap the next one
        is.b = is.nb;
        is.q = 0;
        if (is.b.n > 0) {
            snap_scatter(is, is.nc, g, status, lane);
            is.y = is.ny;
            is.nb = cl.advance(is.b);
            is.nc = load_uvw(uvw, is.nb, lane);
            is.ny = load_vis(vis, is.nb, lane);
        }
    }
    return 1;
}

// Lane 8v + a writes column a of visibility v's tile.
__device__ __forceinline__ void write_tile(ScatterSlot &sl, const float4 *wtab, const float *__restrict__ gwt,
                                           int lane)
{
    const int v = lane >> 3, a = lane & 7;
    if (sl.key[v] < 0)
        return;
    const int fw = sl.fw[v];
    const float4 gw = wtab ? wtab[fw] : __ldg(reinterpret_cast<const float4 *>(gwt) + fw);
    const float gu = reinterpret_cast<const float *>(&sl.rows[v][0][0])[a];
    const float4 v0 = sl.rows[v][1][0], v1 = sl.rows[v][1][1];
    const float gv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
    const float2 y = sl.y[v];
#pragma unroll
    for (int b = 0; b < kUV; ++b) {
        const float2 t = __fmul2_rn(make_float2(gu, gu), __fmul2_rn(y, make_float2(gv[b], gv[b])));
        const float2 c0 = __fmul2_rn(t, make_float2(gw.x, gw.x)), c1 = __fmul2_rn(t, make_float2(gw.y, gw.y));
        const float2 c2 = __fmul2_rn(t, make_float2(gw.z, gw.z)), c3 = __fmul2_rn(t, make_float2(gw.w, gw.w));
        float4 *dst = reinterpret_cast<float4 *>(&sl.tile[v][b][8 * a]);
        dst[0] = make_float4(c0.x, c0.y, c1.x, c1.y);
        dst[1] = make_float4(c2.x, c2.y, c3.x, c3.y);
    }
}

__device__ __forceinline__ void reduce_add_tile(const CUtensorMap *map, uint32_t src, int x, int y)
{
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group"
                 " [%0, {%1, %2}], [%3];"
                 ::"l"(map), "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(kSWarps * kWarp, 1)
grid_scatter_kernel(const Geometry g, const __grid_constant__ CUtensorMap omap,
                    const double *__restrict__ uvw, const float2 *__restrict__ vis_in,
                    const float *__restrict__ guv, const float *__restrict__ gwt, const Schedule sched,
                    DeviceStatus *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ScatterSlot *slots = reinterpret_cast<ScatterSlot *>(smem_raw + wtable_bytes(g)) + (threadIdx.x >> 5) * 2;
    const float4 *wtab = load_wtable(g, gwt, smem_raw);
    const int lane = threadIdx.x & 31;

    pdl_wait();                             // the chunk table (and the zeroed output) are complete
    ClaimerT<kBatch> cl(sched, lane,
                        Prefetch{uvw, 3 * (int)sizeof(double), vis_in, (int)sizeof(float2)});
    ScatterIssue is;
    is.q = 0;
    is.b = cl.claim();
    is.key = -1;
    is.fw = is.fu = is.fv = is.bx = is.by = 0;
    is.y = is.ny = make_float2(0.f, 0.f);
    is.nb = Batch{0, 0, 0, 0};
    is.nc = Coords3{0.0, 0.0, 0.0};
    if (is.b.n > 0) {
        snap_scatter(is, load_uvw(uvw, is.b, lane), g, status, lane);
        is.y = load_vis(vis_in, is.b, lane);
        is.nb = cl.advance(is.b);
        is.nc = load_uvw(uvw, is.nb, lane);
        is.ny = load_vis(vis_in, is.nb, lane);
    }
    int issued = issue_scatter(is, slots[0], cl, guv, uvw, vis_in, g, status, lane);
    for (int done = 0; done < issued; ++done) {
        ScatterSlot &sl = slots[done & 1];
        issued += issue_scatter(is, slots[(done + 1) & 1], cl, guv, uvw, vis_in, g, status, lane);
        cp_async_wait<1>();                 // this lane's row copies of stage `done`
        bulk_wait_read<1>();                // the reduce of stage done - 2 has read this slot's tiles
        __syncwarp();
        write_tile(sl, wtab, gwt, lane);
        fence_proxy_async();                // the tiles, written by the generic proxy, go to the copy engine
        __syncwarp();
        const int v = lane >> 3;
        if ((lane & 7) == 0 && v < sl.n && sl.key[v] >= 0)
            reduce_add_tile(&omap, smem_u32(&sl.tile[v][0][0]), sl.bx[v], sl.by[v]);
        bulk_commit();
        __syncwarp();
    }
    cp_async_wait<0>();
    bulk_wait_all();                        // every reduce has finished before the warp ends
}

}  // namespace
}  // namespace dg

int dg_scatter_warps() { return dg::kSWarps; }

cudaError_t dg_launch_scatter(degrid_plan *p, cudaStream_t st, int n_subgrids, const double *uvw,
                              const float *vis_in, float *sub_out, int grid_blocks)
{
    using namespace dg;
    Schedule sched{p->chunks, p->n_chunks, p->work_counter};
    const size_t smem = wtable_bytes_host(p->geo) + sizeof(ScatterSlot) * 2 * (size_t)kSWarps;
    static std::atomic<size_t> smem_table[kMaxDevices];
    {
        const cudaError_t e = dg_open_smem(dg_smem_record(smem_table, p->device), grid_scatter_kernel, smem);
        if (e != cudaSuccess)
            return e;
    }
    // the output stack as a 2D tensor [S * ny rows][2 nx nz floats]; a box is one footprint
    CUtensorMap map;
    cudaError_t e = encode_2d(&map, sub_out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2 * (uint64_t)p->geo.row_stride,
                              (uint64_t)n_subgrids * p->geo.ny, 8 * (uint64_t)p->geo.row_stride,
                              (uint32_t)(2 * kUV * kW), (uint32_t)kUV);
    if (e != cudaSuccess)
        return e;
    return launch_pdl(grid_scatter_kernel, dim3(grid_blocks), dim3(kSWarps * kWarp), smem, st, p->geo, map, uvw,
                      reinterpret_cast<const float2 *>(vis_in), (const float *)p->guv, (const float *)p->gw,
                      sched, p->status);
}
