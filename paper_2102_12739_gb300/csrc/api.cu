// Host side of the C ABI declared in include/degrid.h: plan management,
// argument validation, scratch management and kernel launches.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "internal.cuh"

cudaError_t dg_launch_pack(cudaStream_t st, dg_dtype dtype, int n_subgrids, int64_t elems,
                           const float *in, void *codes_out, float *scale_out, int sm_count);

namespace {

// Makes `device` current for the duration of an API call and restores the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int device)
    {
        ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

int log2_exact(int x)
{
    if (x <= 0 || (x & (x - 1)) != 0)
        return -1;
    int k = 0;
    while ((1 << k) != x)
        ++k;
    return k;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

dg_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess)
        return DG_OK;
    if (e == cudaErrorMemoryAllocation)
        return DG_ERR_OOM;
    return DG_ERR_CUDA;
}

template <typename T>
dg_status dev_alloc(T **p, size_t n)
{
    *p = nullptr;
    if (n == 0)
        n = 1;
    return from_cuda(cudaMalloc((void **)p, sizeof(T) * n));
}

void free_events(degrid_plan *p)
{
    for (int i = 0; i < p->n_slots; ++i) {
        if (p->ev_start && p->ev_start[i])
            cudaEventDestroy(p->ev_start[i]);
        if (p->ev_stop && p->ev_stop[i])
            cudaEventDestroy(p->ev_stop[i]);
    }
    free(p->ev_start);
    free(p->ev_stop);
    p->ev_start = p->ev_stop = nullptr;
    p->n_slots = 0;
    p->timed_launches = 0;
}

void free_plan_buffers(degrid_plan *p)
{
    free_events(p);
    dg_free_host_exec(p);
    cudaFree(p->guv);
    cudaFree(p->guv2);
    cudaFree(p->gw);
    cudaFree(p->status);
    cudaFree(p->work_counter);
    cudaFree(p->n_chunks);
    cudaFree(p->prefix);
    cudaFree(p->chunks);
}

// Resident warps a call's chunk size is matched to (16 per SM).
constexpr int kCallWarpsPerSm = 16;

// Chunk size of one call: the plan's, halved for small calls until the
// list makes about two chunks per resident warp (so that a short list still
// spreads over the GPU), but never below one 64-visibility pipeline step.
// Results do not depend on it (every visibility's arithmetic is the same).
int call_chunk_for(int sm_count, int plan_chunk, int64_t n_vis)
{
    const int64_t warps = (int64_t)sm_count * kCallWarpsPerSm;
    int c = plan_chunk;
    while (c > 64 && c % 64 == 0 && n_vis / c < 2 * warps)
        c >>= 1;
    return c;
}

int call_chunk(const degrid_plan *p, int64_t n_vis) { return call_chunk_for(p->sm_count, p->chunk, n_vis); }

// Work items the chunk table reserves for calls of up to S subgrids and
// n_vis visibilities: the most that any such call needs, whatever chunk
// call_chunk_for picks for it.  A chunk c below the plan's is picked only
// when the halving test held at 2c, i.e. for n < 4 * warps * c visibilities,
// so the items of that chunk are bounded at min(n_vis, 4 * warps * c - 1).
// Each term grows with S and n_vis, so the reserve does too: a call never
// needs more items than one with larger sizes reserved before it (so a call
// captured in a CUDA graph after a call with larger sizes never allocates).
int64_t reserve_items(int sm_count, int plan_chunk, int S, int64_t n_vis)
{
    int64_t need = dg_schedule_capacity(S, n_vis, plan_chunk, dg_small_items(plan_chunk));
    const int64_t warps = (int64_t)sm_count * kCallWarpsPerSm;
    for (int c = plan_chunk; c > 64 && c % 64 == 0;) {
        c >>= 1;
        const int64_t bound = 4 * warps * c - 1;
        const int64_t n = n_vis < bound ? n_vis : bound;
        const int64_t k = dg_schedule_capacity(S, n, c, dg_small_items(c));
        if (k > need)
            need = k;
    }
    return need;
}

// Grows the schedule scratch so that every call of up to S subgrids and
// n_vis visibilities fits (reserve_items).  This allocates, so it must not
// run inside a stream capture: a first call with sizes at least as large
// has to happen before capturing.
dg_status ensure_capacity(degrid_plan *p, int S, int64_t n_vis, int chunk)
{
    (void)chunk;
    const int64_t need_chunks = reserve_items(p->sm_count, p->chunk, S, n_vis);
    if (need_chunks > 0x7fffffff)
        return DG_ERR_ARG;
    if (S > p->cap_subgrids) {
        cudaDeviceSynchronize();
        cudaFree(p->prefix);
        p->prefix = nullptr;
        p->cap_subgrids = 0;
        dg_status st = dev_alloc(&p->prefix, (size_t)S + 1);
        if (st != DG_OK)
            return st;
        p->cap_subgrids = S;
    }
    if (need_chunks > p->cap_chunks) {
        cudaDeviceSynchronize();
        cudaFree(p->chunks);
        p->chunks = nullptr;
        p->cap_chunks = 0;
        dg_status st = dev_alloc(&p->chunks, (size_t)need_chunks);
        if (st != DG_OK)
            return st;
        p->cap_chunks = (int)need_chunks;
    }
    return DG_OK;
}

// Event pair around the main kernel of a call when timing is enabled.
struct KernelTimer {
    degrid_plan *p;
    cudaStream_t s;
    int slot;
    KernelTimer(degrid_plan *plan, cudaStream_t st) : p(plan), s(st), slot(-1)
    {
        if (p->n_slots > 0) {
            slot = (int)(p->timed_launches % p->n_slots);
            cudaEventRecord(p->ev_start[slot], s);
        }
    }
    void stop()
    {
        if (slot >= 0) {
            cudaEventRecord(p->ev_stop[slot], s);
            p->timed_launches += 1;
        }
    }
};

// The gather and scatter kernels address the stack as one 2D tensor of
// n_subgrids * ny rows with 32-bit row coordinates; past that the plan takes
// the footprint-cache kernels (the same results, bit for bit).
bool tma_rows_fit(const degrid_plan *p, int n_subgrids)
{
    return (int64_t)n_subgrids * p->geo.ny <= (int64_t)0x7fffffff;
}

// Persistent grid: the resident CTAs of every SM, but no more CTAs than
// there are chunks for their chunk-claiming warps.
int grid_blocks(degrid_plan *p, int S, int64_t n_vis, int chunk, int max_per_sm, int claimers_per_block)
{
    int per_sm = p->blocks_per_sm > 0 ? p->blocks_per_sm : max_per_sm;
    if (per_sm < 1)
        per_sm = 1;
    if (per_sm > max_per_sm)
        per_sm = max_per_sm;
    int64_t blocks = (int64_t)p->sm_count * per_sm;
    const int64_t max_chunks = dg_schedule_capacity(S, n_vis, chunk, dg_small_items(chunk));
    const int64_t useful = (max_chunks + claimers_per_block - 1) / claimers_per_block;
    if (blocks > useful)
        blocks = useful;
    return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

extern "C" {

const char *degrid_status_string(dg_status status)
{
    switch (status) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_CUDA: return "CUDA runtime error";
    case DG_ERR_OOM: return "device allocation failed";
    case DG_ERR_DTYPE: return "unsupported storage type or missing scale";
    case DG_ERR_OFFSETS: return "malformed vis_offsets";
    case DG_ERR_UNSUPPORTED: return "unsupported GCF support or subgrid shape";
    case DG_ERR_SCRATCH_LIMIT: return "sizes exceed the fixed scratch of degrid_execute_noalloc";
    case DG_ERR_TIMEOUT: return "a bounded device-side wait gave up; results are incomplete";
    case DG_ERR_BOUNDS: return "an index check of the bounds-checking build failed";
    }
    return "unknown status";
}

const char *degrid_version(void) { return "gb300-degrid 0.1 (sm_103a)"; }

dg_status degrid_schedule_reserve(int sm_count, int plan_chunk, int n_subgrids, int64_t n_vis,
                                  int *call_chunk_out, int64_t *items_out)
{
    if (sm_count < 1 || plan_chunk < dg::kWarp || plan_chunk % dg::kWarp != 0 || plan_chunk > 65536 ||
        n_subgrids < 0 || n_vis < 0)
        return DG_ERR_ARG;
    if (call_chunk_out)
        *call_chunk_out = call_chunk_for(sm_count, plan_chunk, n_vis);
    if (items_out)
        *items_out = reserve_items(sm_count, plan_chunk, n_subgrids, n_vis);
    return DG_OK;
}

// Plan creation for either a separable G_uv table g_uv [O][8] or a 2D one
// g_uv2 [O][O][8][8] (exactly one of them non-null).
static dg_status plan_create(degrid_plan_t *out, int nx, int ny, int nz, const double *g_uv,
                      const double *g_uv2, int uv_support, int uv_oversample, const double *g_w,
                      int w_support, int w_oversample, dg_dtype dtype, int device)
{
    NvtxRange nvtx_range("degrid_plan_create");
    if (!out)
        return DG_ERR_ARG;
    *out = nullptr;
    if ((!g_uv && !g_uv2) || !g_w || nx <= 0 || ny <= 0 || nz <= 0 || device < 0)
        return DG_ERR_ARG;
    if (g_uv2 && (uv_oversample < 1 || uv_oversample > DG_TABLE2D_MAX_OVERSAMPLE))
        return DG_ERR_ARG;
    if (dtype != DG_C64 && dtype != DG_C32_F16 && dtype != DG_C32_BF16)
        return DG_ERR_DTYPE;
    if (uv_support != dg::kUV || w_support != dg::kW)
        return DG_ERR_UNSUPPORTED;
    if (nx < uv_support || ny < uv_support || nz < w_support)
        return DG_ERR_UNSUPPORTED;
    if ((int64_t)nx * ny * nz >= ((int64_t)1 << 31))
        return DG_ERR_UNSUPPORTED;
    const int l2uv = log2_exact(uv_oversample), l2w = log2_exact(w_oversample);
    if (l2uv < 0 || l2w < 0 || l2uv > 20 || l2w > 20)
        return DG_ERR_ARG;
    // every valid oversampled coordinate p = rint(q * O) < n * O must fit 31 bits
    if (((int64_t)(nx > ny ? nx : ny) << l2uv) > ((int64_t)1 << 31) || ((int64_t)nz << l2w) > ((int64_t)1 << 31))
        return DG_ERR_UNSUPPORTED;

    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device >= n_dev)
        return DG_ERR_CUDA;
    DeviceGuard guard(device);
    if (!guard.ok)
        return DG_ERR_CUDA;

    degrid_plan *p = new (std::nothrow) degrid_plan();
    if (!p)
        return DG_ERR_OOM;
    memset(p, 0, sizeof(*p));
    p->device = device;
    if (cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete p;
        return DG_ERR_CUDA;
    }
    p->geo.nx = nx;
    p->geo.ny = ny;
    p->geo.nz = nz;
    p->geo.log2_uv_os = l2uv;
    p->geo.log2_w_os = l2w;
    p->geo.row_stride = nx * nz;
    p->geo.plane = (int64_t)nx * ny * nz;
    // small w tables (16 bytes per row) live in each CTA's shared memory
    p->geo.w_table_rows = (size_t)w_oversample * w_support * sizeof(float) <= 8 * 1024 ? w_oversample : 0;
    p->uv_oversample = uv_oversample;
    p->w_oversample = w_oversample;
    p->dtype = dtype;
    p->chunk = 256;
    p->warps_per_block = dg_max_warps_per_block();
    p->blocks_per_sm = 0;
    p->direct_runs = DG_DIRECT_RUNS_DEFAULT;
    p->host_direct = 1;

    dg_status st = DG_OK;
    const size_t n_uv = g_uv2 ? (size_t)uv_oversample * uv_oversample * uv_support * uv_support
                              : (size_t)uv_oversample * uv_support;
    const double *src_uv = g_uv2 ? g_uv2 : g_uv;
    std::vector<float> h_uv(n_uv), h_w((size_t)w_oversample * w_support);
    for (size_t i = 0; i < h_uv.size(); ++i)
        h_uv[i] = (float)src_uv[i];          // round to nearest
    for (size_t i = 0; i < h_w.size(); ++i)
        h_w[i] = (float)g_w[i];
    float **dst_uv = g_uv2 ? &p->guv2 : &p->guv;
    if ((st = dev_alloc(dst_uv, h_uv.size())) != DG_OK ||
        (st = dev_alloc(&p->gw, h_w.size())) != DG_OK ||
        (st = dev_alloc(&p->status, 1)) != DG_OK ||
        (st = dev_alloc(&p->work_counter, 1)) != DG_OK ||
        (st = dev_alloc(&p->n_chunks, 1)) != DG_OK) {
        free_plan_buffers(p);
        delete p;
        return st;
    }
    cudaError_t e = cudaMemcpy(*dst_uv, h_uv.data(), sizeof(float) * h_uv.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->gw, h_w.data(), sizeof(float) * h_w.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(p->status, 0, sizeof(dg::DeviceStatus));
    if (e == cudaSuccess)
        e = cudaMemset(p->work_counter, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemset(p->n_chunks, 0, sizeof(int));
    if (e != cudaSuccess) {
        free_plan_buffers(p);
        delete p;
        return from_cuda(e);
    }
    *out = p;
    return DG_OK;
}

dg_status degrid_plan_create(degrid_plan_t *out, int nx, int ny, int nz, const double *g_uv,
                             int uv_support, int uv_oversample, const double *g_w,
                             int w_support, int w_oversample, dg_dtype dtype, int device)
{
    return plan_create(out, nx, ny, nz, g_uv, nullptr, uv_support, uv_oversample, g_w, w_support,
                       w_oversample, dtype, device);
}

dg_status degrid_plan_create_2d(degrid_plan_t *out, int nx, int ny, int nz, const double *g_uv2,
                                int uv_oversample, const double *g_w, int w_support, int w_oversample,
                                dg_dtype dtype, int device)
{
    if (!g_uv2) {
        if (out)
            *out = nullptr;
        return DG_ERR_ARG;
    }
    return plan_create(out, nx, ny, nz, nullptr, g_uv2, dg::kUV, uv_oversample, g_w, w_support,
                       w_oversample, dtype, device);
}

void degrid_plan_destroy(degrid_plan_t p)
{
    if (!p)
        return;
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    free_plan_buffers(p);
    delete p;
}

dg_status degrid_plan_set_tuning(degrid_plan_t p, int chunk, int warps_per_block, int blocks_per_sm)
{
    if (!p)
        return DG_ERR_ARG;
    if (chunk > 0 && (chunk % dg::kWarp != 0 || chunk > 65536))
        return DG_ERR_ARG;
    if (warps_per_block > dg_max_warps_per_block())
        return DG_ERR_ARG;
    if (blocks_per_sm > 64)
        return DG_ERR_ARG;
    if (chunk > 0 && chunk != p->chunk) {
        p->chunk = chunk;
        p->cap_chunks = 0;          // chunk table is re-sized on the next call
        DeviceGuard guard(p->device);
        cudaDeviceSynchronize();
        cudaFree(p->chunks);
        p->chunks = nullptr;
    }
    if (warps_per_block > 0 && warps_per_block != p->warps_per_block) {
        p->warps_per_block = warps_per_block;
        p->max_blocks_degrid = p->max_blocks_adjoint = 0;     // occupancy changes
    }
    if (blocks_per_sm >= 0)
        p->blocks_per_sm = blocks_per_sm;
    return DG_OK;
}

dg_status degrid_plan_set_compensated(degrid_plan_t p, int enabled)
{
    if (!p || (enabled != 0 && enabled != 1))
        return DG_ERR_ARG;
    if (enabled != p->compensated) {
        p->compensated = enabled;
        p->max_blocks_degrid = 0;               // another kernel instance
    }
    return DG_OK;
}

dg_status degrid_plan_set_direct_runs(degrid_plan_t p, int min_runs)
{
    if (!p || min_runs < 1 || min_runs > DG_DIRECT_RUNS_NEVER)
        return DG_ERR_ARG;
    if ((min_runs < DG_DIRECT_RUNS_NEVER) != (p->direct_runs < DG_DIRECT_RUNS_NEVER))
        p->max_blocks_degrid = 0;               // another kernel instance
    p->direct_runs = min_runs;
    return DG_OK;
}

dg_status degrid_plan_set_gather(degrid_plan_t p, int enabled)
{
    if (!p || (enabled != 0 && enabled != 1))
        return DG_ERR_ARG;
    if (enabled && !dg_gather_supported(p))
        return DG_ERR_UNSUPPORTED;
    p->gather = enabled;
    return DG_OK;
}

dg_status degrid_plan_set_host_direct(degrid_plan_t p, int enabled)
{
    if (!p || (enabled != 0 && enabled != 1))
        return DG_ERR_ARG;
    p->host_direct = enabled;
    return DG_OK;
}

dg_status degrid_plan_get_host_direct(degrid_plan_t p, int *enabled)
{
    if (!p || !enabled)
        return DG_ERR_ARG;
    *enabled = p->host_direct;
    return DG_OK;
}

dg_status degrid_plan_get_gather(degrid_plan_t p, int *enabled)
{
    if (!p || !enabled)
        return DG_ERR_ARG;
    *enabled = p->gather;
    return DG_OK;
}

dg_status degrid_plan_get_direct_runs(degrid_plan_t p, int *min_runs)
{
    if (!p || !min_runs)
        return DG_ERR_ARG;
    *min_runs = p->direct_runs;
    return DG_OK;
}

dg_status degrid_plan_get_compensated(degrid_plan_t p, int *enabled)
{
    if (!p || !enabled)
        return DG_ERR_ARG;
    *enabled = p->compensated;
    return DG_OK;
}

dg_status degrid_plan_get_tuning(degrid_plan_t p, int *chunk, int *warps_per_block, int *blocks_per_sm)
{
    if (!p)
        return DG_ERR_ARG;
    if (chunk)
        *chunk = p->chunk;
    if (warps_per_block)
        *warps_per_block = p->warps_per_block;
    if (blocks_per_sm)
        *blocks_per_sm = p->blocks_per_sm;
    return DG_OK;
}

dg_status degrid_plan_enable_timing(degrid_plan_t p, int n_slots)
{
    if (!p || n_slots < 0 || n_slots > (1 << 20))
        return DG_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    cudaDeviceSynchronize();
    free_events(p);
    if (n_slots == 0)
        return DG_OK;
    p->ev_start = (cudaEvent_t *)calloc((size_t)n_slots, sizeof(cudaEvent_t));
    p->ev_stop = (cudaEvent_t *)calloc((size_t)n_slots, sizeof(cudaEvent_t));
    if (!p->ev_start || !p->ev_stop) {
        free(p->ev_start);
        free(p->ev_stop);
        p->ev_start = p->ev_stop = nullptr;
        return DG_ERR_OOM;
    }
    p->n_slots = n_slots;
    for (int i = 0; i < n_slots; ++i) {
        if (cudaEventCreate(&p->ev_start[i]) != cudaSuccess ||
            cudaEventCreate(&p->ev_stop[i]) != cudaSuccess) {
            free_events(p);
            return DG_ERR_CUDA;
        }
    }
    return DG_OK;
}

dg_status degrid_plan_kernel_times_ms(degrid_plan_t p, float *ms_out, int capacity, int *count)
{
    if (!p || !count || capacity < 0 || (capacity > 0 && !ms_out))
        return DG_ERR_ARG;
    *count = 0;
    if (p->n_slots == 0 || p->timed_launches == 0)
        return DG_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    long long n = p->timed_launches < p->n_slots ? p->timed_launches : p->n_slots;
    if (n > capacity)
        n = capacity;
    const long long first = p->timed_launches - n;
    cudaError_t e = cudaEventSynchronize(p->ev_stop[(p->timed_launches - 1) % p->n_slots]);
    for (long long k = 0; e == cudaSuccess && k < n; ++k) {
        const int slot = (int)((first + k) % p->n_slots);
        e = cudaEventElapsedTime(ms_out + k, p->ev_start[slot], p->ev_stop[slot]);
    }
    if (e != cudaSuccess)
        return from_cuda(e);
    *count = (int)n;
    return DG_OK;
}

dg_status degrid_execute(degrid_plan_t p, void *stream, int n_subgrids, const void *subgrids,
                         const float *subgrid_scale, const double *uvw,
                         const int64_t *vis_offsets, int64_t n_vis, float *vis_out)
{
    NvtxRange nvtx_range("degrid_execute");
    if (!p || n_subgrids < 0 || n_vis < 0 || !vis_offsets)
        return DG_ERR_ARG;
    if (n_vis > 0 && (!uvw || !vis_out || !subgrids || n_subgrids == 0))
        return DG_ERR_ARG;
    if (n_vis > 0 && p->dtype != DG_C64 && !subgrid_scale)
        return DG_ERR_DTYPE;
    if (!aligned(uvw, 8) || !aligned(vis_out, 8) || !aligned(vis_offsets, 8) ||
        !aligned(subgrids, 16) || !aligned(subgrid_scale, 4))
        return DG_ERR_ARG;
    if (n_vis == 0)
        return DG_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    const int chunk = call_chunk(p, n_vis);
    dg_status st = ensure_capacity(p, n_subgrids, n_vis, chunk);
    if (st != DG_OK)
        return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = dg::launch_schedule(s, vis_offsets, n_subgrids, n_vis, chunk, dg_small_items(chunk),
                                        p->prefix, p->n_chunks, p->chunks, p->cap_chunks, p->work_counter,
                                        p->status);
    if (e != cudaSuccess)
        return from_cuda(e);
    if (p->gather && tma_rows_fit(p, n_subgrids)) {
        // one CTA per SM
        const int blocks = grid_blocks(p, n_subgrids, n_vis, chunk, 1, dg_gather_warps(p->dtype));
        KernelTimer timer(p, s);
        e = dg_launch_gather(p, s, subgrids, n_subgrids, subgrid_scale, uvw, vis_out, blocks);
        timer.stop();
        return from_cuda(e);
    }
    if (p->max_blocks_degrid == 0)
        p->max_blocks_degrid = dg_max_blocks_per_sm_degrid(p);
    const int blocks = grid_blocks(p, n_subgrids, n_vis, chunk, p->max_blocks_degrid, p->warps_per_block);
    KernelTimer timer(p, s);
    e = dg_launch_degrid(p, s, subgrids, subgrid_scale, uvw, vis_offsets, vis_out, blocks);
    timer.stop();
    return from_cuda(e);
}

dg_status grid_adjoint_execute(degrid_plan_t p, void *stream, int n_subgrids, const double *uvw,
                               const int64_t *vis_offsets, int64_t n_vis, const float *vis_in,
                               float *sub_out, int accumulate)
{
    NvtxRange nvtx_range("grid_adjoint_execute");
    if (!p || n_subgrids < 0 || n_vis < 0 || !vis_offsets)
        return DG_ERR_ARG;
    if (n_subgrids > 0 && !sub_out)
        return DG_ERR_ARG;
    if (n_vis > 0 && (!uvw || !vis_in || n_subgrids == 0))
        return DG_ERR_ARG;
    if (!aligned(uvw, 8) || !aligned(vis_in, 8) || !aligned(vis_offsets, 8) || !aligned(sub_out, 8))
        return DG_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (!accumulate && n_subgrids > 0) {
        cudaError_t e = cudaMemsetAsync(sub_out, 0, sizeof(float) * 2 * (size_t)p->geo.plane * n_subgrids, s);
        if (e != cudaSuccess)
            return from_cuda(e);
    }
    if (n_vis == 0)
        return DG_OK;
    const int chunk = call_chunk(p, n_vis);
    dg_status st = ensure_capacity(p, n_subgrids, n_vis, chunk);
    if (st != DG_OK)
        return st;
    cudaError_t e = dg::launch_schedule(s, vis_offsets, n_subgrids, n_vis, chunk, dg_small_items(chunk),
                                        p->prefix, p->n_chunks, p->chunks, p->cap_chunks, p->work_counter,
                                        p->status);
    if (e != cudaSuccess)
        return from_cuda(e);
    if (p->gather && aligned(sub_out, 16) && tma_rows_fit(p, n_subgrids)) {
        // scattered coverage: every visibility's tile added by a tensor reduce, one CTA per SM
        const int blocks = grid_blocks(p, n_subgrids, n_vis, chunk, 1, dg_scatter_warps());
        KernelTimer timer(p, s);
        e = dg_launch_scatter(p, s, n_subgrids, uvw, vis_in, sub_out, blocks);
        timer.stop();
        return from_cuda(e);
    }
    if (p->max_blocks_adjoint == 0)
        p->max_blocks_adjoint = dg_max_blocks_per_sm_adjoint(p);
    const int blocks = grid_blocks(p, n_subgrids, n_vis, chunk, p->max_blocks_adjoint, p->warps_per_block);
    KernelTimer timer(p, s);
    e = dg_launch_adjoint(p, s, uvw, vis_offsets, vis_in, sub_out, blocks);
    timer.stop();
    return from_cuda(e);
}

dg_status degrid_coords_execute(degrid_plan_t p, void *stream, const double *uvw, int64_t n_vis,
                                int32_t *coords_out)
{
    NvtxRange nvtx_range("degrid_coords_execute");
    if (!p || n_vis < 0)
        return DG_ERR_ARG;
    if (n_vis > 0 && (!uvw || !coords_out))
        return DG_ERR_ARG;
    if (!aligned(uvw, 8) || !aligned(coords_out, 4))
        return DG_ERR_ARG;
    if (n_vis == 0)
        return DG_OK;
    DeviceGuard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    return from_cuda(dg_launch_coords(p, (cudaStream_t)stream, uvw, n_vis, coords_out));
}

dg_status degrid_pack_subgrids(void *stream, dg_dtype dtype, int n_subgrids, int64_t elems,
                               const float *in, void *codes_out, float *scale_out)
{
    if (dtype != DG_C32_F16 && dtype != DG_C32_BF16)
        return DG_ERR_DTYPE;
    if (n_subgrids < 0 || n_subgrids > 65535 || elems < 0)
        return DG_ERR_ARG;
    if (n_subgrids > 0 && (!scale_out || (elems > 0 && (!in || !codes_out))))
        return DG_ERR_ARG;
    if (!aligned(in, 4) || !aligned(codes_out, 2) || !aligned(scale_out, 4))
        return DG_ERR_ARG;
    if (n_subgrids == 0)
        return DG_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DG_ERR_CUDA;
    return from_cuda(dg_launch_pack((cudaStream_t)stream, dtype, n_subgrids, elems, in, codes_out,
                                    scale_out, sms));
}

dg_status degrid_get_status(degrid_plan_t p, void *stream, int64_t *n_invalid)
{
    if (!p)
        return DG_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    dg::DeviceStatus h{};
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(&h, p->status, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemset(p->status, 0, sizeof(h));
    if (e != cudaSuccess)
        return from_cuda(e);
    if (n_invalid)
        *n_invalid = (int64_t)h.n_invalid;
    if (h.flags & dg::kFlagTimeout)
        return DG_ERR_TIMEOUT;
    if (h.flags & dg::kFlagBounds)
        return DG_ERR_BOUNDS;
    return (h.flags & (dg::kFlagOffsets | dg::kFlagCapacity)) ? DG_ERR_OFFSETS : DG_OK;
}

}  // extern "C"
