// Auxiliary kernels: the coordinate step on its own (for bit-exact checks of
// the indices and GCF rows used by degrid.cu) and the conversion of complex64
// subgrids to the FP16 / BF16 storage with a per-subgrid scale.
#include "internal.cuh"

namespace dg {
namespace {

// Same device function as the degridding and gridding kernels use.
__global__ void coords_kernel(const Geometry g, const double *__restrict__ uvw, int64_t n_vis,
                              int *__restrict__ out, DeviceStatus *__restrict__ status)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n_vis; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool in = i < n_vis;
        bool valid = false;
        if (in) {
            VisCoords c;
            valid = visibility_coords(__ldg(uvw + 3 * i), __ldg(uvw + 3 * i + 1),
                                      __ldg(uvw + 3 * i + 2), g, c);
            int *o = out + 6 * i;
            o[0] = valid ? c.x0 : -1;
            o[1] = valid ? c.y0 : -1;
            o[2] = valid ? c.z0 : -1;
            o[3] = valid ? c.fu : -1;
            o[4] = valid ? c.fv : -1;
            o[5] = valid ? c.fw : -1;
        }
        const unsigned bad = __ballot_sync(kFull, in && !valid);
        if ((threadIdx.x & 31) == 0 && bad)
            atomicAdd(&status->n_invalid, (unsigned long long)__popc(bad));
    }
}

// scale[s] = max |component| of subgrid s (scale zeroed beforehand).  The
// values are non-negative, so their IEEE bit patterns order like unsigned
// integers and an integer atomicMax finds the float maximum.
__global__ void pack_scale_kernel(const float *__restrict__ in, int64_t comps_per_subgrid,
                                  float *__restrict__ scale)
{
    const int s = blockIdx.y;
    const float *src = in + (int64_t)s * comps_per_subgrid;
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < comps_per_subgrid;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(src[i]));
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1)
        m = fmaxf(m, __shfl_xor_sync(kFull, m, d));
    if ((threadIdx.x & 31) == 0)
        atomicMax(reinterpret_cast<unsigned *>(scale + s), __float_as_uint(m));
}

template <int DT>
__global__ void pack_codes_kernel(const float *__restrict__ in, int64_t comps_per_subgrid,
                                  int64_t n_comps, const float *__restrict__ scale,
                                  unsigned short *__restrict__ codes)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_comps;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float sc = scale[i / comps_per_subgrid];
        const float q = sc > 0.f ? __fdiv_rn(in[i], sc) : 0.f;
        unsigned short bits;
        if (DT == DG_C32_F16)
            bits = __half_as_ushort(__float2half_rn(q));
        else
            bits = __bfloat16_as_ushort(__float2bfloat16_rn(q));
        codes[i] = bits;
    }
}

}  // namespace
}  // namespace dg

cudaError_t dg_launch_coords(degrid_plan *p, cudaStream_t st, const double *uvw,
                             int64_t n_vis, int32_t *coords_out)
{
    using namespace dg;
    if (n_vis == 0)
        return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (n_vis + threads - 1) / threads;
    const int64_t cap = (int64_t)p->sm_count * 8;
    if (blocks > cap)
        blocks = cap;
    coords_kernel<<<(int)blocks, threads, 0, st>>>(p->geo, uvw, n_vis, coords_out, p->status);
    return cudaGetLastError();
}

cudaError_t dg_launch_pack(cudaStream_t st, dg_dtype dtype, int n_subgrids, int64_t elems,
                           const float *in, void *codes_out, float *scale_out, int sm_count)
{
    using namespace dg;
    const int64_t comps = 2 * elems;
    cudaError_t err = cudaMemsetAsync(scale_out, 0, sizeof(float) * (size_t)n_subgrids, st);
    if (err != cudaSuccess || n_subgrids == 0 || elems == 0)
        return err;
    int bx = (int)((comps + 255) / 256);
    const int want = (sm_count * 8 + n_subgrids - 1) / n_subgrids;
    if (bx > want)
        bx = want > 0 ? want : 1;
    pack_scale_kernel<<<dim3(bx, n_subgrids), 256, 0, st>>>(in, comps, scale_out);
    if ((err = cudaGetLastError()) != cudaSuccess)
        return err;
    const int64_t total = comps * n_subgrids;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)sm_count * 16)
        blocks = (int64_t)sm_count * 16;
    auto *codes = reinterpret_cast<unsigned short *>(codes_out);
    if (dtype == DG_C32_F16)
        pack_codes_kernel<DG_C32_F16><<<(int)blocks, 256, 0, st>>>(in, comps, total, scale_out, codes);
    else
        pack_codes_kernel<DG_C32_BF16><<<(int)blocks, 256, 0, st>>>(in, comps, total, scale_out, codes);
    return cudaGetLastError();
}
