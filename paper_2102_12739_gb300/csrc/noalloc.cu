// degrid_execute_noalloc: the degridding call for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: real-time
// pipelines that must not call into the CUDA allocator after start-up
// (cudaMalloc and cudaFree can synchronise the device and stall every other
// stream, which breaks a latency budget), and hosts whose whole device-memory
// budget is owned by another allocator, where a library that allocates on
// its own is not allowed.  degrid_execute_noalloc therefore needs no plan: the
// caller passes the GCF tables and every input and output as device
// pointers, and all scratch the kernels need (the chunk schedule, the work
// counter and the status words) comes from the fixed, file-scope array
// below.  Every GPU that loads the library holds this array
// until the process exits.
#include <mutex>

#include "internal.cuh"

cudaError_t dg_launch_degrid(degrid_plan *p, cudaStream_t st, const void *subgrids,
                             const float *scale, const double *uvw,
                             const int64_t *vis_offsets, float *vis_out, int grid_blocks);

namespace {

// Scratch layout, in bytes from the start of the array.
constexpr int kChunk = 1024;    // visibilities per work item in this entry point
constexpr size_t kMaxChunks =
    ((size_t)DG_NOALLOC_MAX_VIS + kChunk - 1) / kChunk + DG_NOALLOC_MAX_SUBGRIDS + 1;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffChunks = 0;
constexpr size_t kOffPrefix = align256(kOffChunks + kMaxChunks * sizeof(dg::ChunkDesc));
constexpr size_t kOffCounters = align256(kOffPrefix + (DG_NOALLOC_MAX_SUBGRIDS + 1) * sizeof(int));
constexpr size_t kOffStatus = align256(kOffCounters + 2 * sizeof(int));
constexpr size_t kScratchBytes = align256(kOffStatus + sizeof(dg::DeviceStatus));
static_assert(kScratchBytes <= DG_NOALLOC_SCRATCH_BYTES, "no-alloc scratch layout exceeds its array");

// The scratch itself.  In host code `g_scratch` is only a stand-in for the
// symbol, not a device address; the address is looked up per device below.
static __device__ __align__(256) unsigned char g_scratch[DG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_dev[kMaxDevices];      // device address of g_scratch, per device

// Looked up once per device, on the first call made with that device
// current.
dg_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices)
        return DG_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_dev[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr)
            return DG_ERR_CUDA;
        g_scratch_dev[device] = static_cast<unsigned char *>(ptr);
    }
    *out = g_scratch_dev[device];
    return DG_OK;
}

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

dg_status from_cuda(cudaError_t e) { return e == cudaSuccess ? DG_OK : DG_ERR_CUDA; }

}  // namespace

extern "C" dg_status degrid_execute_noalloc(void *stream, int nx, int ny, int nz,
                                            const float *g_uv, int uv_oversample,
                                            const float *g_w, int w_oversample, dg_dtype dtype,
                                            int n_subgrids, const void *subgrids,
                                            const float *subgrid_scale, const double *uvw,
                                            const int64_t *vis_offsets, int64_t n_vis,
                                            float *vis_out, unsigned long long *status_out)
{
    NvtxRange nvtx_range("degrid_execute_noalloc");
    if (nx < 8 || ny < 8 || nz < 4 || (int64_t)nx * ny * nz >= ((int64_t)1 << 31))
        return DG_ERR_ARG;
    if (dtype != DG_C64 && dtype != DG_C32_F16 && dtype != DG_C32_BF16)
        return DG_ERR_DTYPE;
    const int l2uv = log2_exact(uv_oversample), l2w = log2_exact(w_oversample);
    if (l2uv < 0 || l2w < 0 || !g_uv || !g_w || n_subgrids < 0 || n_vis < 0 || !vis_offsets)
        return DG_ERR_ARG;
    if (((int64_t)(nx > ny ? nx : ny) << l2uv) > ((int64_t)1 << 31) || ((int64_t)nz << l2w) > ((int64_t)1 << 31))
        return DG_ERR_ARG;
    if (uv_oversample > DG_NOALLOC_MAX_UV_OVERSAMPLE || w_oversample > DG_NOALLOC_MAX_W_OVERSAMPLE ||
        n_subgrids > DG_NOALLOC_MAX_SUBGRIDS || n_vis > DG_NOALLOC_MAX_VIS)
        return DG_ERR_SCRATCH_LIMIT;
    if (n_vis > 0 && (!uvw || !vis_out || !subgrids || n_subgrids == 0))
        return DG_ERR_ARG;
    if (n_vis > 0 && dtype != DG_C64 && !subgrid_scale)
        return DG_ERR_DTYPE;
    if (!aligned(uvw, 8) || !aligned(vis_out, 8) || !aligned(vis_offsets, 8) ||
        !aligned(subgrids, 16) || !aligned(subgrid_scale, 4) || !aligned(g_uv, 4) ||
        !aligned(g_w, 4) || !aligned(status_out, 8))
        return DG_ERR_ARG;

    int device = 0, sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return DG_ERR_CUDA;
    unsigned char *scratch = nullptr;
    dg_status st = scratch_address(device, &scratch);
    if (st != DG_OK)
        return st;

    // A plan descriptor on the host stack that points into the scratch; the
    // kernels are the ones degrid_execute launches.
    degrid_plan p{};
    p.device = device;
    p.sm_count = sms;
    p.geo.nx = nx;
    p.geo.ny = ny;
    p.geo.nz = nz;
    p.geo.log2_uv_os = l2uv;
    p.geo.log2_w_os = l2w;
    p.geo.row_stride = nx * nz;
    p.geo.plane = (int64_t)nx * ny * nz;
    p.geo.w_table_rows = w_oversample;          // at most 512 rows (8 KiB): staged in shared memory
    p.uv_oversample = uv_oversample;
    p.w_oversample = w_oversample;
    p.dtype = dtype;
    p.guv = const_cast<float *>(g_uv);
    p.gw = const_cast<float *>(g_w);
    p.chunks = reinterpret_cast<dg::ChunkDesc *>(scratch + kOffChunks);
    p.prefix = reinterpret_cast<int *>(scratch + kOffPrefix);
    p.n_chunks = reinterpret_cast<int *>(scratch + kOffCounters);
    p.work_counter = p.n_chunks + 1;
    p.status = status_out ? reinterpret_cast<dg::DeviceStatus *>(status_out)
                          : reinterpret_cast<dg::DeviceStatus *>(scratch + kOffStatus);
    p.cap_subgrids = DG_NOALLOC_MAX_SUBGRIDS;
    p.cap_chunks = (int)kMaxChunks;
    p.chunk = kChunk;
    p.warps_per_block = dg_max_warps_per_block();
    p.blocks_per_sm = 0;
    p.direct_runs = DG_DIRECT_RUNS_DEFAULT;

    cudaStream_t s = (cudaStream_t)stream;
    // The array keeps whatever the previous call left: the status words must
    // start at zero (the scheduler zeroes the work counter itself).
    cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(dg::DeviceStatus), s);
    if (e != cudaSuccess || n_vis == 0)
        return from_cuda(e);
    e = dg::launch_schedule(s, vis_offsets, n_subgrids, n_vis, p.chunk, 0, p.prefix, p.n_chunks,
                            p.chunks, p.cap_chunks, p.work_counter, p.status);
    if (e != cudaSuccess)
        return from_cuda(e);
    int per_sm = dg_max_blocks_per_sm_degrid(&p);
    int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t useful = ((n_vis / kChunk + n_subgrids) + p.warps_per_block - 1) / p.warps_per_block;
    if (blocks > useful)
        blocks = useful;
    if (blocks < 1)
        blocks = 1;
    return from_cuda(dg_launch_degrid(&p, s, subgrids, subgrid_scale, uvw, vis_offsets, vis_out,
                                      (int)blocks));
}
