// FP32 arithmetic peak of the device, measured: the denominator of the
// degridding kernel's roofline.  The footprint sum is bound by FP32
// fused multiply-adds (256 complex x real products per visibility, Section
// "Implementation"), so its roofline is the rate at which the SMs retire
// them.  This kernel fills every SM with independent FMA chains, scalar
// (FFMA) or packed two-wide (FFMA2, the form the degridding kernel issues),
// and the host times it with CUDA events.
#include "internal.cuh"

namespace dg {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 8;         // 2048 threads: every warp slot of the SM
constexpr int kChains = 8;                  // independent chains per thread
constexpr int kUnroll = 16;                 // loop iterations per branch

// acc <- acc * m + a on every chain; m and a are launch arguments, so nothing
// folds.  With m just below 1 and a small the values stay finite and normal.
template <bool kPacked>
__global__ void __launch_bounds__(kPeakThreads)
fp32_peak_kernel(int iters, float m, float a, float *__restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float sum = 0.0f;
    if (kPacked) {
        float2 acc[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            acc[c] = make_float2(1.0f + 0.001f * (float)(t & 7) + 0.01f * c, 1.0f - 0.01f * c);
        const float2 m2 = make_float2(m, m), a2 = make_float2(a, a);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < kChains; ++c)
                    acc[c] = __ffma2_rn(acc[c], m2, a2);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            sum += acc[c].x + acc[c].y;
    } else {
        float acc[2 * kChains];
#pragma unroll
        for (int c = 0; c < 2 * kChains; ++c)
            acc[c] = 1.0f + 0.001f * (float)(t & 7) + 0.01f * c;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int c = 0; c < 2 * kChains; ++c)
                    acc[c] = __fmaf_rn(acc[c], m, a);
        }
#pragma unroll
        for (int c = 0; c < 2 * kChains; ++c)
            sum += acc[c];
    }
    out[t] = sum;
}

}  // namespace
}  // namespace dg

extern "C" dg_status degrid_measure_fp32_peak(int device, int packed, double *tflops)
{
    using namespace dg;
    if (!tflops || device < 0)
        return DG_ERR_ARG;
    *tflops = 0.0;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
        return DG_ERR_CUDA;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * kPeakBlocksPerSM;
    const long long threads = (long long)blocks * kPeakThreads;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess)
        e = cudaMalloc(&out, sizeof(float) * (size_t)threads);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t1);
    // 2 flop per lane FMA; 2 lanes per FFMA2 or two scalar chains per pair
    const int iters = 2048;                 // about 4 ms per launch at 80 TFLOP/s
    const double flop = (double)threads * iters * kUnroll * kChains * 2 * 2;
    float best = 0.0f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {   // launch 0 warms up
        e = cudaEventRecord(t0, st);
        if (e == cudaSuccess) {
            if (packed)
                fp32_peak_kernel<true><<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999999f, 1e-7f, out);
            else
                fp32_peak_kernel<false><<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999999f, 1e-7f, out);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaEventRecord(t1, st);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, t0, t1);
        if (e == cudaSuccess && rep > 0 && ms > 0.0f && (best == 0.0f || ms < best))
            best = ms;
    }
    if (t0)
        cudaEventDestroy(t0);
    if (t1)
        cudaEventDestroy(t1);
    if (st)
        cudaStreamDestroy(st);
    cudaFree(out);
    cudaSetDevice(prev);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    *tflops = flop / (best * 1e-3) / 1e12;
    return DG_OK;
}
