// degrid_execute_host: the degridding call with inputs and output in host
// memory, in one of two ways.
//
// In place (the default when the subgrids, coordinates and output are
// page-locked, i.e. mapped into the GPU's address space): the kernel reads
// the coordinates and the footprint rows it needs straight from host memory
// over the host link and writes the visibilities back the same way; only the
// offsets (and unmapped scales) are copied.  A dense list touches a small
// part of its subgrid (on the 64-line benchmark 1 % of the stack), so the
// link carries the coordinates and little else.
//
// By copies (pageable buffers, a plan with the gather kernel, or in-place
// access disabled): the subgrid stack is split into groups of consecutive
// subgrids (about 64 MB of subgrid data each); for every group the plan's
// three streams run
//   copy-in:   subgrids, coordinates, rebased offsets (and scales) -> slot
//   sums:      degrid_execute on the slot                  (waits copy-in)
//   copy-out:  visibilities slot -> host                   (waits sums)
// through a ring of two device slots, so the copies of group g + 1 and the
// copy-out of group g - 1 overlap the sums of group g.  Groups whose lists
// are empty are skipped without copying their subgrids.
//
// Either way the call returns when the host output is complete.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.cuh"

namespace {

constexpr size_t kGroupBytes = size_t(64) << 20;    // subgrid bytes per group (target)
constexpr int kSlots = 2;

struct Guard {
    int prev = -1;
    bool ok = false;
    explicit Guard(int device) { ok = cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(device) == cudaSuccess; }
    ~Guard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

size_t elem_bytes(dg_dtype t) { return t == DG_C64 ? 8 : 4; }

}  // namespace

// Streams, events and staging owned by a plan once degrid_execute_host ran.
struct dg_host_exec {
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    cudaEvent_t ev_in[kSlots] = {}, ev_run[kSlots] = {}, ev_out[kSlots] = {};
    void *sub[kSlots] = {};
    float *scale[kSlots] = {};
    double *uvw[kSlots] = {};
    int64_t *offs[kSlots] = {};
    float *out[kSlots] = {};
    int cap_subgrids = 0;           // per slot
    int64_t cap_vis = 0;            // per slot
    int64_t *h_offs = nullptr;      // pinned: rebased offsets of every group
    size_t cap_h_offs = 0;
    int64_t *d_offs = nullptr;      // in-place calls: the offsets, and scales if unmapped
    float *d_scale = nullptr;
    int cap_direct = 0;             // subgrids d_offs / d_scale hold
};

void dg_free_host_exec(degrid_plan *p)
{
    dg_host_exec *x = p->hostx;
    if (!x)
        return;
    for (int k = 0; k < kSlots; ++k) {
        cudaFree(x->sub[k]);
        cudaFree(x->scale[k]);
        cudaFree(x->uvw[k]);
        cudaFree(x->offs[k]);
        cudaFree(x->out[k]);
        if (x->ev_in[k])
            cudaEventDestroy(x->ev_in[k]);
        if (x->ev_run[k])
            cudaEventDestroy(x->ev_run[k]);
        if (x->ev_out[k])
            cudaEventDestroy(x->ev_out[k]);
    }
    cudaFree(x->d_offs);
    cudaFree(x->d_scale);
    if (x->s_in)
        cudaStreamDestroy(x->s_in);
    if (x->s_run)
        cudaStreamDestroy(x->s_run);
    if (x->s_out)
        cudaStreamDestroy(x->s_out);
    cudaFreeHost(x->h_offs);
    delete x;
    p->hostx = nullptr;
}

namespace {

cudaError_t create_exec(degrid_plan *p)
{
    dg_host_exec *x = new (std::nothrow) dg_host_exec();
    if (!x)
        return cudaErrorMemoryAllocation;
    p->hostx = x;
    cudaError_t e = cudaStreamCreateWithFlags(&x->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&x->s_run, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&x->s_out, cudaStreamNonBlocking);
    for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&x->ev_in[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&x->ev_run[k], cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&x->ev_out[k], cudaEventDisableTiming);
    }
    return e;
}

// Grows the device slots to `subgrids` subgrids and `vis` visibilities each.
cudaError_t reserve_slots(degrid_plan *p, int subgrids, int64_t vis)
{
    dg_host_exec *x = p->hostx;
    cudaError_t e = cudaSuccess;
    if (subgrids > x->cap_subgrids) {
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
            cudaFree(x->sub[k]);
            cudaFree(x->scale[k]);
            cudaFree(x->offs[k]);
            x->sub[k] = nullptr;
            x->scale[k] = nullptr;
            x->offs[k] = nullptr;
            e = cudaMalloc(&x->sub[k], (size_t)subgrids * p->geo.plane * elem_bytes(p->dtype));
            if (e == cudaSuccess)
                e = cudaMalloc(&x->scale[k], sizeof(float) * (size_t)subgrids);
            if (e == cudaSuccess)
                e = cudaMalloc(&x->offs[k], sizeof(int64_t) * ((size_t)subgrids + 1));
        }
        x->cap_subgrids = e == cudaSuccess ? subgrids : 0;
    }
    if (e == cudaSuccess && vis > x->cap_vis) {
        for (int k = 0; k < kSlots && e == cudaSuccess; ++k) {
            cudaFree(x->uvw[k]);
            cudaFree(x->out[k]);
            x->uvw[k] = nullptr;
            x->out[k] = nullptr;
            e = cudaMalloc(&x->uvw[k], sizeof(double) * 3 * (size_t)vis);
            if (e == cudaSuccess)
                e = cudaMalloc(&x->out[k], sizeof(float) * 2 * (size_t)vis);
        }
        x->cap_vis = e == cudaSuccess ? vis : 0;
    }
    return e;
}

struct Group {
    int s0, n;          // first subgrid, subgrids
    int64_t v0, nv;     // first visibility, visibilities
    size_t h_at;        // position of its rebased offsets in the pinned buffer
};

// Device address under which the GPU reads host buffer h in place:
// page-locked memory mapped into the device's address space; else nullptr.
void *mapped(const void *h)
{
    if (!h)
        return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();             // clear the error of an unknown pointer
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The in-place form: the kernel reads subgrids, coordinates (and mapped
// scales) from host memory and writes the output there.
dg_status execute_in_place(degrid_plan *p, int n_subgrids, const void *sub_d, const float *subgrid_scale,
                           const float *scale_d, const double *uvw_d, const int64_t *vis_offsets,
                           int64_t n_vis, float *out_d)
{
    dg_host_exec *x = p->hostx;
    cudaError_t e = cudaSuccess;
    const bool need_scale = p->dtype != DG_C64 && !scale_d;
    if (n_subgrids > x->cap_direct) {
        cudaFree(x->d_offs);
        cudaFree(x->d_scale);
        x->d_offs = nullptr;
        x->d_scale = nullptr;
        x->cap_direct = 0;
        e = cudaMalloc(&x->d_offs, sizeof(int64_t) * ((size_t)n_subgrids + 1));
        if (e == cudaSuccess)
            e = cudaMalloc(&x->d_scale, sizeof(float) * (size_t)n_subgrids);
        if (e != cudaSuccess)
            return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
        x->cap_direct = n_subgrids;
    }
    e = cudaMemcpyAsync(x->d_offs, vis_offsets, sizeof(int64_t) * ((size_t)n_subgrids + 1),
                        cudaMemcpyHostToDevice, x->s_run);
    if (e == cudaSuccess && need_scale)
        e = cudaMemcpyAsync(x->d_scale, subgrid_scale, sizeof(float) * (size_t)n_subgrids,
                            cudaMemcpyHostToDevice, x->s_run);
    if (e != cudaSuccess)
        return DG_ERR_CUDA;
    p->host_inputs = 1;
    const dg_status st = degrid_execute(p, x->s_run, n_subgrids, sub_d,
                                        p->dtype == DG_C64 ? nullptr : (need_scale ? x->d_scale : scale_d),
                                        uvw_d, x->d_offs, n_vis, out_d);
    p->host_inputs = 0;
    e = cudaStreamSynchronize(x->s_run);
    if (st != DG_OK)
        return st;
    return e == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

}  // namespace

extern "C" dg_status degrid_execute_host(degrid_plan_t p, int n_subgrids, const void *subgrids,
                                         const float *subgrid_scale, const double *uvw,
                                         const int64_t *vis_offsets, int64_t n_vis, float *vis_out)
{
    NvtxRange nvtx_range("degrid_execute_host");
    if (!p || n_subgrids < 0 || n_vis < 0 || !vis_offsets)
        return DG_ERR_ARG;
    if (n_vis > 0 && (!uvw || !vis_out || !subgrids || n_subgrids == 0))
        return DG_ERR_ARG;
    if (n_vis > 0 && p->dtype != DG_C64 && !subgrid_scale)
        return DG_ERR_DTYPE;
    // the offsets are on the host: check them here
    if (vis_offsets[0] != 0 || vis_offsets[n_subgrids] != n_vis)
        return DG_ERR_OFFSETS;
    for (int s = 0; s < n_subgrids; ++s)
        if (vis_offsets[s + 1] < vis_offsets[s])
            return DG_ERR_OFFSETS;
    if (n_vis == 0)
        return DG_OK;

    Guard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    if (!p->hostx) {
        const cudaError_t ce = create_exec(p);
        if (ce != cudaSuccess) {
            dg_free_host_exec(p);
            return ce == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
        }
    }
    if (p->host_direct && !p->gather) {
        void *sub_d = mapped(subgrids), *uvw_d = mapped(uvw), *out_d = mapped(vis_out);
        if (sub_d && uvw_d && out_d)
            return execute_in_place(p, n_subgrids, sub_d, subgrid_scale,
                                    static_cast<const float *>(mapped(subgrid_scale)),
                                    static_cast<const double *>(uvw_d), vis_offsets, n_vis,
                                    static_cast<float *>(out_d));
    }

    const size_t sub_bytes = (size_t)p->geo.plane * elem_bytes(p->dtype);
    const int per_group = (int)std::max<size_t>(1, std::min<size_t>(kGroupBytes / sub_bytes, (size_t)n_subgrids));
    std::vector<Group> groups;
    size_t h_need = 0;
    int max_n = 0;
    int64_t max_nv = 0;
    for (int s0 = 0; s0 < n_subgrids; s0 += per_group) {
        const int n = std::min(per_group, n_subgrids - s0);
        const int64_t nv = vis_offsets[s0 + n] - vis_offsets[s0];
        if (nv == 0)
            continue;                       // nothing to degrid: no copies
        groups.push_back(Group{s0, n, vis_offsets[s0], nv, h_need});
        h_need += (size_t)n + 1;
        max_n = std::max(max_n, n);
        max_nv = std::max(max_nv, nv);
    }

    cudaError_t e = cudaSuccess;
    dg_host_exec *x = p->hostx;
    e = reserve_slots(p, max_n, max_nv);
    if (e == cudaSuccess && h_need > x->cap_h_offs) {
        cudaFreeHost(x->h_offs);
        x->h_offs = nullptr;
        x->cap_h_offs = 0;
        e = cudaMallocHost(&x->h_offs, sizeof(int64_t) * h_need);
        if (e == cudaSuccess)
            x->cap_h_offs = h_need;
    }
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    for (const Group &gr : groups)
        for (int k = 0; k <= gr.n; ++k)
            x->h_offs[gr.h_at + k] = vis_offsets[gr.s0 + k] - gr.v0;

    dg_status st = DG_OK;
    const char *sub_h = static_cast<const char *>(subgrids);
    for (size_t g = 0; g < groups.size() && st == DG_OK && e == cudaSuccess; ++g) {
        const Group &gr = groups[g];
        const int k = (int)(g % kSlots);
        if (g >= (size_t)kSlots)            // the slot's previous copy-out has finished
            e = cudaStreamWaitEvent(x->s_in, x->ev_out[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x->sub[k], sub_h + (size_t)gr.s0 * sub_bytes, (size_t)gr.n * sub_bytes,
                                cudaMemcpyHostToDevice, x->s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x->uvw[k], uvw + 3 * gr.v0, sizeof(double) * 3 * (size_t)gr.nv,
                                cudaMemcpyHostToDevice, x->s_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x->offs[k], x->h_offs + gr.h_at, sizeof(int64_t) * ((size_t)gr.n + 1),
                                cudaMemcpyHostToDevice, x->s_in);
        if (e == cudaSuccess && p->dtype != DG_C64)
            e = cudaMemcpyAsync(x->scale[k], subgrid_scale + gr.s0, sizeof(float) * (size_t)gr.n,
                                cudaMemcpyHostToDevice, x->s_in);
        if (e == cudaSuccess)
            e = cudaEventRecord(x->ev_in[k], x->s_in);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(x->s_run, x->ev_in[k], 0);
        if (e != cudaSuccess)
            break;
        st = degrid_execute(p, x->s_run, gr.n, x->sub[k], p->dtype != DG_C64 ? x->scale[k] : nullptr,
                            x->uvw[k], x->offs[k], gr.nv, x->out[k]);
        if (st != DG_OK)
            break;
        e = cudaEventRecord(x->ev_run[k], x->s_run);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(x->s_out, x->ev_run[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vis_out + 2 * gr.v0, x->out[k], sizeof(float) * 2 * (size_t)gr.nv,
                                cudaMemcpyDeviceToHost, x->s_out);
        if (e == cudaSuccess)
            e = cudaEventRecord(x->ev_out[k], x->s_out);
    }
    const cudaError_t e_in = cudaStreamSynchronize(x->s_in);
    const cudaError_t e_run = cudaStreamSynchronize(x->s_run);
    const cudaError_t e_out = cudaStreamSynchronize(x->s_out);
    if (st != DG_OK)
        return st;
    if (e != cudaSuccess || e_in != cudaSuccess || e_run != cudaSuccess || e_out != cudaSuccess)
        return DG_ERR_CUDA;
    return DG_OK;
}
