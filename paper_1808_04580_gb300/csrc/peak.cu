// Measured arithmetic rates of the current GPU: the denominators of the
// ALU rooflines the spread and gather are bound by.  Not a paper construct.
//
// Every thread keeps 16 FP32 lanes (16 scalar registers, or 8 packed pairs
// for fma.rn.f32x2) or 8 FP64 registers and updates each with a dependent
// chain of fused multiply-adds whose multiplier and addend are kernel
// arguments, so nothing folds at compile time; with 64 resident warps per SM
// the chains hide the pipe latency.  The accumulators are stored only when
// their sum equals an impossible value, which keeps the work live without
// memory traffic.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace nfl {

constexpr int kRateThreads = 256;
constexpr int kRateBlocksPerSm = 8;   // 2048 threads per SM

__global__ void __launch_bounds__(kRateThreads) fma_rate_f32(int iters, float b, float c, float *sink) {
    float a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = threadIdx.x * 1e-3f + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    if (s == -1.2345e-30f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kRateThreads) fma_rate_f32x2(int iters, float b, float c, float *sink) {
    unsigned long long a[8];
    unsigned long long bb, cc;
    asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
    asm("mov.b64 %0, {%1, %2};" : "=l"(cc) : "f"(c), "f"(c));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float lo = threadIdx.x * 1e-3f + 2 * k, hi = lo + 1.f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a[k]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(bb), "l"(cc));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a[k]));
        s += lo + hi;
    }
    if (s == -1.2345e-30f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kRateThreads) fma_rate_f64(int iters, double b, double c, float *sink) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(b), "d"(c));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -1.2345e-300) sink[threadIdx.x] = float(s);
}

}  // namespace nfl

extern "C" nfl_status nfl_fma_rate(int kind, void *stream, double *flops_per_s, double *ms_out) {
    if (kind < NFL_RATE_FP32_FMA || kind > NFL_RATE_FP64_FMA || !flops_per_s) return NFL_ERR_INVALID_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NFL_ERR_CUDA;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto release = [&]() {
        cudaFree(sink);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&sink, nfl::kRateThreads * sizeof(float)) != cudaSuccess) return NFL_ERR_OUT_OF_MEMORY;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        release();
        return NFL_ERR_CUDA;
    }
    const int blocks = sms * nfl::kRateBlocksPerSm;
    // about 4 ms per launch at the expected rates (FP64 is far slower on this part)
    const int iters = kind == NFL_RATE_FP64_FMA ? 256 : 16384;
    const double fma_per_thread = 16.0 * iters / (kind == NFL_RATE_FP64_FMA ? 2.0 : 1.0);
    const double flops = 2.0 * fma_per_thread * nfl::kRateThreads * blocks;
    auto launch = [&]() {
        if (kind == NFL_RATE_FP32_FMA)
            nfl::fma_rate_f32<<<blocks, nfl::kRateThreads, 0, s>>>(iters, 0.999f, 1e-3f, sink);
        else if (kind == NFL_RATE_FP32X2_FMA)
            nfl::fma_rate_f32x2<<<blocks, nfl::kRateThreads, 0, s>>>(iters, 0.999f, 1e-3f, sink);
        else
            nfl::fma_rate_f64<<<blocks, nfl::kRateThreads, 0, s>>>(iters, 0.999, 1e-3, sink);
        return cudaGetLastError();
    };
    float best = 1e30f;
    nfl_status st = NFL_OK;
    for (int r = 0; r < 6 && st == NFL_OK; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess || launch() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) {
            st = NFL_ERR_CUDA;
            break;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = NFL_ERR_CUDA;
        if (r > 0) best = std::min(best, t);   // the first launch warms up
    }
    release();
    if (st != NFL_OK) return st;
    *flops_per_s = flops / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return NFL_OK;
}
