// Arithmetic peak of the GPU for the roofline of the formal solver, measured
// rather than derived: kernels of independent fused multiply-add chains
// (FP32 FFMA, packed FP32 FFMA2 on float2 pairs, FP64 DFMA) timed with CUDA
// events. The paper has no counterpart; the sweep's roofline is bound by plain
// FP32 arithmetic issue, whose peak this measures.
#include <cuda_runtime.h>

#include <algorithm>

#include "porta.h"

namespace {

constexpr int kChains = 8;       // independent accumulators per thread (covers the FMA latency)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) fma_f32_kernel(int iters, float a, float b, float *out)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_f32x2_kernel(int iters, float a, float b, float *out)
{
    float2 x[kChains];
    const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2(threadIdx.x * 1e-3f + c, c * 0.5f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], av, bv);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma_f64_kernel(int iters, double a, double b, double *out)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int porta_fma_peak(int kind, double seconds, double *tflops, double *total_ms)
{
    if (kind < 0 || kind > 2 || !(seconds > 0) || !tflops) return PORTA_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PORTA_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PORTA_ECUDA;
    const int blocks = sms * 8;   // 64 warps per SM
    void *out = nullptr;
    // a few MB of device memory for the results (the library's only allocation outside a context)
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(double)) != cudaSuccess) return PORTA_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a contraction factor just below 1 keeps every chain finite
    const float af = 0.9999999f, bf = 1e-7f;
    const double ad = 0.9999999999, bd = 1e-10;
    auto launch = [&](int iters) {
        if (kind == 0) fma_f32_kernel<<<blocks, kThreads>>>(iters, af, bf, (float *)out);
        else if (kind == 1) fma_f32x2_kernel<<<blocks, kThreads>>>(iters, af, bf, (float *)out);
        else fma_f64_kernel<<<blocks, kThreads>>>(iters, ad, bd, (double *)out);
    };
    // flops per launch: 2 per FMA, 2 FMAs per packed FFMA2
    const double per_iter = 2.0 * kChains * (kind == 1 ? 2 : 1) * (double)blocks * kThreads;
    int iters = 1 << 12;
    double best = 0.0, spent = 0.0;
    int rc = PORTA_OK;
    launch(iters);   // warm-up
    while (spent < 1e3 * seconds) {
        cudaEventRecord(e0);
        launch(iters);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = PORTA_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        spent += ms;
        best = std::max(best, per_iter * iters / (ms * 1e-3) / 1e12);
        if (ms < 50.f && iters < (1 << 26)) iters *= 2;   // grow launches to tens of ms
    }
    if (cudaGetLastError() != cudaSuccess) rc = PORTA_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *tflops = best;
    if (total_ms) *total_ms = spent;
    return rc;
}
