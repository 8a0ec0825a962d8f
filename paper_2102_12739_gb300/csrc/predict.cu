// The step upstream of degridding: the subgrid stack itself.
//
// The paper starts from "pre-computed grid data" of the improved w-stacking
// method (Introduction) and does not describe how it is made.  Following
// improved w-stacking (Ye, Gull, Tan & Nikolic 2020), the grid at a w-plane
// w_c is the Fourier transform of the sky image after the image-plane
// correction of the gridding kernels (a real taper T) and the w-phase screen
// of the plane:
//   G[s][y][x][c] = sum_{b,a} I[b][a] T[b][a]
//                   exp(-2 pi i ((x - N/2 + u0_s)(a - N/2) / N + (y - N/2 + v0_s)(b - N/2) / N
//                                 + (w0_s + c dw_s)(n_ab - 1))),
// n_ab = sqrt(1 - l_a^2 - m_b^2), l_a = (a - N/2) theta / N; pixels with
// l^2 + m^2 >= 1 contribute nothing.  A subgrid is an N x N window of cells
// at nz consecutive w-planes, stored [y][x][c] like the stack the degridding
// kernels read.
//
// Per pass of up to P subgrids, three steps on the caller's stream:
//  1. screen_kernel (hand-written): for every pixel and subgrid, the tapered
//     image times the w-phase screen of each plane and (-1)^(a + b) into a
//     work buffer [P][nz][N][N].  The phase w (n - 1) runs to hundreds of
//     turns, far beyond FP32's resolution, and FP64 runs at a small fraction
//     of the FP32 rate on this part, so it is reduced to a fraction of a turn
//     in double-float arithmetic: w and n - 1 are each held as an unevaluated
//     sum of two floats (hi + lo, split in FP64 once per subgrid and once per
//     pixel), the product hi * hi and its exact rounding error come from one
//     multiply and one FMA, the whole turns are removed from the product
//     exactly, and the small terms are added after (about 3e-8 turns of
//     error for |w (n - 1)| < 2^22 turns).  The fraction goes through FP32
//     sincospif; planes after the first are rotated by the plane step's
//     screen.
//  2. a batched 2D FFT of the P * nz planes (cuFFT, in place);
//  3. window_kernel (hand-written): the cell window of each subgrid -- an
//     integer offset (u0, v0) is a cyclic shift of the transform -- times
//     (-1)^(kx + ky), which together with step 1's factor makes the plain
//     FFT the centred transform above (N even), interleaved into the
//     [y][x][c] layout with 16-byte stores.
#include <cufft.h>
#include <math.h>

#include <new>

#include "internal.cuh"

struct subgrid_predict_plan {
    int device;
    int n, nz, per_pass;
    cufftHandle fft;
    bool fft_ok;
    float2 *work;       // [per_pass][nz][n][n]
    float2 *nm1;        // [n][n]: n - 1 per pixel as (hi, lo) floats, hi NaN outside the unit circle
};

namespace {

constexpr int kThreads = 256;

// n - 1 for every pixel, in the cancellation-free form -r^2 / (1 + sqrt(1 - r^2)),
// as the unevaluated sum hi + lo of two floats.
__global__ void nm1_kernel(float2 *__restrict__ nm1, int n, double dl)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= n)
        return;
    const int i = b * n + a;
    const double l = (double)(a - n / 2) * dl, m = (double)(b - n / 2) * dl;
    const double r2 = l * l + m * m;
    if (r2 < 1.0) {
        const double v = -r2 / (1.0 + sqrt(1.0 - r2));
        const float hi = (float)v;
        nm1[i] = make_float2(hi, (float)(v - (double)hi));
    } else {
        nm1[i] = make_float2(__int_as_float(0x7fc00000), 0.f);
    }
}

// exp(-2 pi i w (n - 1)) with w = (w_hi + w_lo) and n - 1 = (n_hi + n_lo):
// the turns of the product are reduced to [-1/2, 1/2] in double-float
// arithmetic (|w (n - 1)| < 2^22 turns), then rotated in FP32.
__device__ __forceinline__ float2 screen_phasor(float w_hi, float w_lo, float2 nm)
{
    const float p = w_hi * nm.x;
    const float e = fmaf(w_hi, nm.x, -p);                   // p + e = w_hi * n_hi exactly
    const float c = fmaf(w_hi, nm.y, w_lo * nm.x);          // cross terms (w_lo * n_lo dropped)
    const float f = (p - rintf(p)) + (e + c);               // p - rint(p) is exact
    float s, co;
    sincospif(2.0f * f, &s, &co);
    return make_float2(co, -s);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Step 1: grid (ceil(N / kThreads), N rows); thread (a, b) makes pixel (a, b)
// of every subgrid of the pass, so the image, taper and n - 1 of the pixel
// are read once per pass, and the plane step's screen is reused while
// consecutive subgrids have the same plane spacing (bit for bit the value it
// would compute again).  The subgrids' w0 and dw are split into (hi, lo)
// floats by the block, 256 subgrids at a time.  32-bit index arithmetic
// throughout (the plan keeps N * N * nz below 2^31).
__global__ void __launch_bounds__(kThreads)
screen_kernel(const float2 *__restrict__ image, const float *__restrict__ taper, const float2 *__restrict__ nm1,
              const double *__restrict__ w_planes, int first, int count, int n, int nz, float2 *__restrict__ work)
{
    __shared__ float4 wsplit[kThreads];     // per subgrid: (w0 hi, w0 lo, dw hi, dw lo)
    const int a = blockIdx.x * kThreads + threadIdx.x, b = blockIdx.y;
    const bool in = a < n;
    const int i = b * n + (in ? a : 0);
    const int np = n * n;
    const float2 nm = in ? nm1[i] : make_float2(0.f, 0.f);
    const bool lit = in && !isnan(nm.x);
    float2 base = make_float2(0.f, 0.f);
    if (lit) {
        const float2 v = image[i];
        const float t = (taper ? taper[i] : 1.f) * (((a + b) & 1) ? -1.f : 1.f);
        base = make_float2(v.x * t, v.y * t);
    }
    float2 step = make_float2(1.f, 0.f);
    float dw_hi = 0.f, dw_lo = 0.f;
    bool have_step = false;
    for (int t0 = 0; t0 < count; t0 += kThreads) {
        __syncthreads();                    // the previous tile's splits are no longer read
        if (t0 + (int)threadIdx.x < count) {
            const int64_t s = first + t0 + (int64_t)threadIdx.x;
            const double w0 = w_planes[2 * s], dw = w_planes[2 * s + 1];
            const float w0h = (float)w0, dwh = (float)dw;
            wsplit[threadIdx.x] = make_float4(w0h, (float)(w0 - (double)w0h), dwh, (float)(dw - (double)dwh));
        }
        __syncthreads();
        const int tn = count - t0 < kThreads ? count - t0 : kThreads;
        for (int k = 0; k < tn; ++k) {
            const float4 ws = wsplit[k];
            float2 cur = make_float2(0.f, 0.f);
            if (lit) {
                cur = cmul(base, screen_phasor(ws.x, ws.y, nm));
                if (!have_step || ws.z != dw_hi || ws.w != dw_lo) {
                    step = screen_phasor(ws.z, ws.w, nm);
                    dw_hi = ws.z;
                    dw_lo = ws.w;
                    have_step = true;
                }
            }
            if (in) {
                float2 *out = work + (int64_t)(t0 + k) * nz * np + i;
                for (int c = 0; c < nz; ++c) {
                    out[(int64_t)c * np] = cur;
                    cur = cmul(cur, lit ? step : make_float2(1.f, 0.f));
                }
            }
        }
    }
}

// Step 3: grid (ceil(N / kThreads), N rows, subgrids of the pass).
__global__ void __launch_bounds__(kThreads)
window_kernel(const float2 *__restrict__ work, const int32_t *__restrict__ uv_offsets, int first, int n, int nz,
              float2 *__restrict__ sub_out)
{
    __shared__ int off[2];                  // the subgrid's cell offsets reduced to [0, n)
    const int sp = blockIdx.z, s = first + sp;
    if (threadIdx.x < 2) {
        const int o = uv_offsets[2 * (int64_t)s + threadIdx.x] % n;     // |o| < n: no overflow below
        off[threadIdx.x] = o < 0 ? o + n : o;
    }
    __syncthreads();
    const int x = blockIdx.x * kThreads + threadIdx.x, y = blockIdx.y;
    if (x >= n)
        return;
    const int u0 = off[0], v0 = off[1];
    const int kx = x + u0 < n ? x + u0 : x + u0 - n, ky = y + v0 < n ? y + v0 : y + v0 - n;
    const float sg = ((kx + ky) & 1) ? -1.f : 1.f;
    const int np = n * n;
    const float2 *src = work + (int64_t)sp * nz * np + ky * n + kx;
    float2 *dst = sub_out + ((int64_t)s * np + (int64_t)y * n + x) * nz;
    if ((nz & 1) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        for (int c = 0; c < nz; c += 2) {
            const float2 p = src[(int64_t)c * np], q = src[(int64_t)(c + 1) * np];
            *reinterpret_cast<float4 *>(dst + c) = make_float4(p.x * sg, p.y * sg, q.x * sg, q.y * sg);
        }
    } else {
        for (int c = 0; c < nz; ++c) {
            const float2 p = src[(int64_t)c * np];
            dst[c] = make_float2(p.x * sg, p.y * sg);
        }
    }
}

dg_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess)
        return DG_OK;
    return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

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

void free_plan(subgrid_predict_plan *p)
{
    if (p->fft_ok)
        cufftDestroy(p->fft);
    cudaFree(p->work);
    cudaFree(p->nm1);
}

}  // namespace

extern "C" {

dg_status subgrid_predict_plan_create(subgrid_predict_plan_t *out, int n, int nz, int subgrids_per_pass,
                                      int device)
{
    NvtxRange nvtx_range("subgrid_predict_plan_create");
    if (!out)
        return DG_ERR_ARG;
    *out = nullptr;
    if (n < 8 || n % 2 != 0 || (int64_t)n * n * nz >= ((int64_t)1 << 31) || nz < 1 || nz > 64 ||
        subgrids_per_pass < 1 || subgrids_per_pass > 4096 || device < 0)
        return DG_ERR_ARG;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device >= n_dev)
        return DG_ERR_CUDA;
    DeviceGuard guard(device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    subgrid_predict_plan *p = new (std::nothrow) subgrid_predict_plan();
    if (!p)
        return DG_ERR_OOM;
    p->device = device;
    p->n = n;
    p->nz = nz;
    p->per_pass = subgrids_per_pass;
    p->fft_ok = false;
    p->work = nullptr;
    p->nm1 = nullptr;
    const size_t np = (size_t)n * n;
    cudaError_t e = cudaMalloc((void **)&p->work, sizeof(float2) * np * nz * subgrids_per_pass);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&p->nm1, sizeof(float2) * np);
    if (e == cudaSuccess)           // planes a short last pass leaves unwritten hold zeros
        e = cudaMemset(p->work, 0, sizeof(float2) * np * nz * subgrids_per_pass);
    if (e != cudaSuccess) {
        free_plan(p);
        delete p;
        return from_cuda(e);
    }
    int dims[2] = {n, n};
    if (cufftPlanMany(&p->fft, 2, dims, nullptr, 1, (int)np, nullptr, 1, (int)np, CUFFT_C2C,
                      nz * subgrids_per_pass) != CUFFT_SUCCESS) {
        free_plan(p);
        delete p;
        return DG_ERR_CUDA;
    }
    p->fft_ok = true;
    *out = p;
    return DG_OK;
}

void subgrid_predict_plan_destroy(subgrid_predict_plan_t p)
{
    if (!p)
        return;
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    free_plan(p);
    delete p;
}

dg_status subgrid_predict_execute(subgrid_predict_plan_t p, void *stream, double theta, const float *image,
                                  const float *taper, int n_subgrids, const int32_t *uv_offsets,
                                  const double *w_planes, float *subgrids_out)
{
    NvtxRange nvtx_range("subgrid_predict_execute");
    if (!p || n_subgrids < 0 || !(theta > 0.0) || !isfinite(theta))
        return DG_ERR_ARG;
    if (n_subgrids == 0)
        return DG_OK;
    if (!image || !uv_offsets || !w_planes || !subgrids_out)
        return DG_ERR_ARG;
    if ((uintptr_t)image % 8 || (uintptr_t)taper % 4 || (uintptr_t)uv_offsets % 4 || (uintptr_t)w_planes % 8 ||
        (uintptr_t)subgrids_out % 8)
        return DG_ERR_ARG;
    DeviceGuard guard(p->device);
    if (!guard.ok)
        return DG_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t np = (int64_t)p->n * p->n;
    nm1_kernel<<<dim3((unsigned)((p->n + kThreads - 1) / kThreads), (unsigned)p->n), kThreads, 0, st>>>(
        p->nm1, p->n, theta / p->n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return from_cuda(e);
    if (cufftSetStream(p->fft, st) != CUFFT_SUCCESS)
        return DG_ERR_CUDA;
    const float2 *img = reinterpret_cast<const float2 *>(image);
    float2 *out = reinterpret_cast<float2 *>(subgrids_out);
    const unsigned row_blocks = (unsigned)((p->n + kThreads - 1) / kThreads);
    for (int first = 0; first < n_subgrids; first += p->per_pass) {
        const int count = n_subgrids - first < p->per_pass ? n_subgrids - first : p->per_pass;
        const dim3 grid(row_blocks, (unsigned)p->n, (unsigned)count);
        screen_kernel<<<dim3(row_blocks, (unsigned)p->n), kThreads, 0, st>>>(img, taper, p->nm1, w_planes, first,
                                                                             count, p->n, p->nz, p->work);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return from_cuda(e);
        // the whole batch (planes past `count` hold earlier passes' values and are not read)
        if (cufftExecC2C(p->fft, reinterpret_cast<cufftComplex *>(p->work), reinterpret_cast<cufftComplex *>(p->work),
                         CUFFT_FORWARD) != CUFFT_SUCCESS)
            return DG_ERR_CUDA;
        window_kernel<<<grid, kThreads, 0, st>>>(p->work, uv_offsets, first, p->n, p->nz, out);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return from_cuda(e);
    }
    return DG_OK;
}

}  // extern "C"
