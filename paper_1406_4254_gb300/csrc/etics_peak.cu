// etics_peak.cu -- arithmetic-rate microbenchmark that supplies the
// denominators of the roofline fractions: how many FP32 and FP64 fused
// multiply-adds per second this GPU completes when nothing else limits it.
// The paper compares single- and double-precision speed of its kernels
// (Sec. 3.4); this measures the two rates themselves.
//
// Every thread runs kChains independent accumulator chains (enough
// independent work per warp to cover the FMA latency), each step
// a <- a * b + c with b and c kernel arguments (nothing folds at compile
// time), and writes one value at the end so the work cannot be elided.
#include "etics_internal.h"

namespace etics {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 16;
constexpr int kInner = 16;   // unrolled steps per loop trip

__global__ void __launch_bounds__(kPeakThreads) ffma_peak_kernel(int64_t iters, float b, float c,
                                                                 float* sink) {
    float a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the paired FP32 FMA of Blackwell (one instruction, two lanes' worth of
// FMAs per thread): kChains / 2 float2 chains, the same FMA count
__global__ void __launch_bounds__(kPeakThreads) ffma2_peak_kernel(int64_t iters, float b, float c,
                                                                  float* sink) {
    float2 a[kChains / 2];
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j)
        a[j] = make_float2((float)(threadIdx.x + 2 * j) * 1e-3f,
                           (float)(threadIdx.x + 2 * j + 1) * 1e-3f);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u)
#pragma unroll
            for (int j = 0; j < kChains / 2; ++j) a[j] = __ffma2_rn(a[j], b2, c2);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) s += a[j].x + a[j].y;
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) dfma_peak_kernel(int64_t iters, double b, double c,
                                                                 float* sink) {
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = (double)(threadIdx.x + j) * 1e-3;
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kInner; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

}  // namespace

int fma_peak(int kind, int blocks, int64_t iters, float* sink, double* flops,
             const LaunchCtx& ctx) {
    // b slightly below 1 and c small keep every chain finite and normal
    const float b = 0.9999999f, c = 1e-7f;
    if (kind == ETICS_PEAK_FFMA)
        ffma_peak_kernel<<<blocks, kPeakThreads, 0, ctx.stream>>>(iters, b, c, sink);
    else if (kind == ETICS_PEAK_FFMA2)
        ffma2_peak_kernel<<<blocks, kPeakThreads, 0, ctx.stream>>>(iters, b, c, sink);
    else
        dfma_peak_kernel<<<blocks, kPeakThreads, 0, ctx.stream>>>(iters, 0.9999999999, 1e-13,
                                                                  sink);
    if (cudaGetLastError() != cudaSuccess) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    *flops = 2.0 * kChains * kInner * (double)iters * kPeakThreads * (double)blocks;
    return ETICS_OK;
}

}  // namespace etics
