// Device peaks measured on the GPU, the denominators of the degridding
// roofline and its diagnostics.
//  * FP32 FMA rate: the footprint sum is bound by FP32 fused multiply-adds
//    (256 complex x real products per visibility, Section "Implementation"),
//    so its roofline is the rate at which the SMs retire them.  A kernel
//    fills every SM with independent FMA chains, scalar (FFMA) or packed
//    two-wide (FFMA2, the form the degridding kernel issues).
//  * L2 read bandwidth: without footprint reuse every visibility gathers its
//    own 8 x 8 x 4 footprint (2 KB complex64, 1 KB FP16/BF16) from L2.  A
//    kernel streams an L2-resident buffer into every SM with L1-bypassing
//    16-byte loads.
//  * L2 reduce-add rate: gridding of scattered coverage adds every
//    visibility's 2 KB footprint tile into the stack with one tensor
//    reduce-add of the copy engine (scatter.cu).  A kernel has one lane of
//    every warp issue such reduce-adds (boxes of 8 rows x 256 bytes at
//    pseudo-random footprint positions of an L2-resident stack) back to back.
// The host times them with CUDA events (best of 5 launches after a warm-up).
#include "tma.cuh"

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

constexpr int kL2PerThread = 8;             // 16-byte loads per thread per pass

// Reads buf[0, n4) `passes` times, grid-strided, bypassing L1; the xor of
// everything read is stored so that no load is dead.
__global__ void __launch_bounds__(kPeakThreads)
l2_read_kernel(const uint4 *__restrict__ buf, long long n4, int passes, unsigned *__restrict__ out)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned acc = 0;
    for (int p = 0; p < passes; ++p) {
#pragma unroll 4
        for (long long i = t; i < n4; i += stride) {
            const uint4 x = __ldcg(buf + i);
            acc ^= x.x ^ x.y ^ x.z ^ x.w;
        }
    }
    out[t] = acc;
}

constexpr int kRedWarps = 16;                // warps per CTA, one CTA per SM
constexpr int kRedCols = 2048;              // floats per row of the stack (a 512 x 4 complex64 row)
constexpr int kRedBoxW = 64;                // floats per box row: one footprint row (8 x 4 complex64)
constexpr int kRedBoxH = 8;                 // box rows

// Every warp's lane 0 issues `iters` tensor reduce-adds of its 2 KB tile into
// the stack at pseudo-random footprint positions (x on a 4-sample boundary,
// as a footprint's is), keeping up to 4 in flight.
__global__ void __launch_bounds__(kRedWarps * kWarp, 1)
l2_reduce_kernel(const __grid_constant__ CUtensorMap map, int rows, int iters)
{
    __shared__ __align__(128) float tile[kRedWarps][kRedBoxH][kRedBoxW];
    for (int i = threadIdx.x; i < kRedWarps * kRedBoxH * kRedBoxW; i += blockDim.x)
        (&tile[0][0][0])[i] = 1e-30f;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane != 0)
        return;
    unsigned h = (blockIdx.x * kRedWarps + w) * 2654435761u + 12345u;
    const uint32_t src = (uint32_t)__cvta_generic_to_shared(&tile[w][0][0]);
    for (int i = 0; i < iters; ++i) {
        h = h * 1664525u + 1013904223u;
        const int x = (int)((h >> 8) % (unsigned)(kRedCols / 8 - kRedBoxW / 8 + 1)) * 8;
        const int y = (int)((h >> 3) % (unsigned)(rows - kRedBoxH + 1));
        asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group"
                     " [%0, {%1, %2}], [%3];" ::"l"(&map), "r"(x), "r"(y), "r"(src) : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory");
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Times `launch` (a callable issuing one launch on `st`): best of 5 after a
// warm-up; returns the best duration in ms (0 on error, with *err set).
template <class F>
float best_of_5(cudaStream_t st, F launch, cudaError_t *err)
{
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&t1);
    float best = 0.0f;
    for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {   // launch 0 warms up
        e = cudaEventRecord(t0, st);
        if (e == cudaSuccess) {
            launch();
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
    *err = e;
    return best;
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
    if (e == cudaSuccess)
        e = cudaMalloc(&out, sizeof(float) * (size_t)threads);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // 2 flop per lane FMA; 2 lanes per FFMA2 or two scalar chains per pair
    const int iters = 2048;                 // about 4 ms per launch at 80 TFLOP/s
    const double flop = (double)threads * iters * kUnroll * kChains * 2 * 2;
    float best = 0.0f;
    if (e == cudaSuccess)
        best = best_of_5(st, [&] {
            if (packed)
                fp32_peak_kernel<true><<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999999f, 1e-7f, out);
            else
                fp32_peak_kernel<false><<<blocks, kPeakThreads, 0, st>>>(iters, 0.9999999f, 1e-7f, out);
        }, &e);
    if (st)
        cudaStreamDestroy(st);
    cudaFree(out);
    cudaSetDevice(prev);
    if (e != cudaSuccess || best <= 0.0f)
        return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    *tflops = flop / (best * 1e-3) / 1e12;
    return DG_OK;
}

extern "C" dg_status degrid_measure_l2_read_bw(int device, double *gbs)
{
    using namespace dg;
    if (!gbs || device < 0)
        return DG_ERR_ARG;
    *gbs = 0.0;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
        return DG_ERR_CUDA;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = sms * kPeakBlocksPerSM;
    const long long threads = (long long)blocks * kPeakThreads;
    const long long n4 = threads * kL2PerThread;           // 39.8 MB on 152 SMs: L2-resident
    const int passes = 1000;
    uint4 *buf = nullptr;
    unsigned *out = nullptr;
    cudaStream_t st = nullptr;
    if (e == cudaSuccess)
        e = cudaMalloc(&buf, sizeof(uint4) * (size_t)n4);
    if (e == cudaSuccess)
        e = cudaMalloc(&out, sizeof(unsigned) * (size_t)threads);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(buf, 1, sizeof(uint4) * (size_t)n4, st);
    float best = 0.0f;
    if (e == cudaSuccess)
        best = best_of_5(st, [&] {
            l2_read_kernel<<<blocks, kPeakThreads, 0, st>>>(buf, n4, passes, out);
        }, &e);
    if (st)
        cudaStreamDestroy(st);
    cudaFree(out);
    cudaFree(buf);
    cudaSetDevice(prev);
    if (e != cudaSuccess || best <= 0.0f)
        return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    *gbs = (double)passes * (double)n4 * sizeof(uint4) / (best * 1e-3) / 1e9;
    return DG_OK;
}

extern "C" dg_status degrid_measure_l2_reduce_bw(int device, double *gbs)
{
    using namespace dg;
    if (!gbs || device < 0)
        return DG_ERR_ARG;
    *gbs = 0.0;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
        return DG_ERR_CUDA;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int rows = 2048;                  // 16 MB stack: L2-resident
    const int iters = 4096;
    float *buf = nullptr;
    cudaStream_t st = nullptr;
    CUtensorMap map;
    if (e == cudaSuccess)
        e = cudaMalloc(&buf, sizeof(float) * (size_t)rows * kRedCols);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(buf, 0, sizeof(float) * (size_t)rows * kRedCols, st);
    if (e == cudaSuccess)
        e = encode_2d(&map, buf, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, kRedCols, rows, sizeof(float) * kRedCols,
                      kRedBoxW, kRedBoxH);
    float best = 0.0f;
    if (e == cudaSuccess)
        best = best_of_5(st, [&] { l2_reduce_kernel<<<sms, kRedWarps * kWarp, 0, st>>>(map, rows, iters); }, &e);
    if (st)
        cudaStreamDestroy(st);
    cudaFree(buf);
    cudaSetDevice(prev);
    if (e != cudaSuccess || best <= 0.0f)
        return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
    const double bytes = (double)sms * kRedWarps * iters * kRedBoxH * kRedBoxW * sizeof(float);
    *gbs = bytes / (best * 1e-3) / 1e9;
    return DG_OK;
}
