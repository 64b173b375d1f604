// Device helpers shared by the spread and gather kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace nfl {

// Normalized Kaiser-Bessel window phi(delta) / phi(0) at grid offset delta,
// |delta| <= m:  (m / s) sinh(b s) / sinh(b m),  s = sqrt(m^2 - delta^2).
// Written as  exp(-b delta^2 / (s + m)) * m * (1 - e^{-2 b s}) / (s (1 - e^{-2 b m}))
// because b (s - m) = -b delta^2 / (s + m) has no cancellation: forming
// sinh(b s) / sinh(b m) directly in FP32 turns the rounding of b into a
// relative bias of b m ulp (~2e-6) shared by every weight.  The limit at
// s = 0 is 2 b m e^{-b m} / (1 - e^{-2 b m}).  phi(0) is put back into the
// Fourier multiplier.  inv_den = 1 / (1 - e^{-2 b m}).
template <typename T>
__device__ __forceinline__ T kb_weight(T delta, T m, T b, T inv_den);

template <>
__device__ __forceinline__ double kb_weight<double>(double delta, double m, double b, double inv_den) {
    double s2 = m * m - delta * delta;
    s2 = s2 > 0.0 ? s2 : 0.0;
    const double s = sqrt(s2);
    const double head = exp(-b * delta * delta / (s + m));
    const double tail = s > 0.0 ? -expm1(-2.0 * b * s) / s : 2.0 * b;
    return head * m * tail * inv_den;
}

// FP32: single-precision functions only (the FP64 pipe of this GPU is narrow).
// The head factor carries the weight's magnitude and uses the accurate expf;
// the tail (1 - e^{-2bs})/s differs from 1/s only where s is small, i.e. where
// the weight is ~e^{-bm} relative to its peak, so fast intrinsics suffice there.
template <>
__device__ __forceinline__ float kb_weight<float>(float delta, float m, float b, float inv_den) {
    float s2 = fmaf(-delta, delta, m * m);
    s2 = s2 > 0.f ? s2 : 0.f;
    const float s = s2 > 0.f ? s2 * rsqrtf(s2) : 0.f;
    const float head = expf(-__fdividef(b * delta * delta, s + m));
    const float tail = s > 1e-4f ? __fdividef(1.f - __expf(-2.f * b * s), s) : 2.f * b;
    return head * m * tail * inv_den;
}

// Two FP32 lanes in one 64-bit register: lane 0 in the low half.
// w rounded to the nearest BF16 value (ties to even), returned in FP32: the
// window taps of the BF16W form.
__device__ __forceinline__ float round_bf16(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lane_of(unsigned long long v, int hi) {
    return __uint_as_float(static_cast<unsigned>(hi ? (v >> 32) : v));
}
// a * b + c on both lanes.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// a * b on both lanes.
__device__ __forceinline__ unsigned long long fmul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// 2^k with k the largest integer such that sum|x~| * 2^k < 2^62 (FP32C fixed point).
__device__ __forceinline__ double fixed_scale_of(double abs_sum) {
    if (!(abs_sum > 0.0)) return 1.0;
    int e;
    frexp(abs_sum, &e);
    int k = 62 - e;
    k = k > 120 ? 120 : (k < -120 ? -120 : k);     // 2^k stays a normal FP32 number
    return ldexp(1.0, k);
}

// FP32 value (already scaled by 2^k, |v| < 2^62) -> nearest int64 with 32-bit
// conversions only.  |v| = h 2^32 + l with h = floor(|v| 2^-32) and
// 0 <= l < 2^32: both parts are exact in FP32 (power-of-two scaling; l keeps
// a subset of the bits of |v|), and the sign is applied to the integer.
__device__ __forceinline__ long long to_fixed(float v) {
    const float av = fabsf(v);
    const float hf = floorf(av * 2.3283064365386963e-10f);
    const float lf = fmaf(hf, -4294967296.0f, av);
    const unsigned long long mag = ((unsigned long long)__float2uint_rn(hf) << 32) + __float2uint_rn(lf);
    return v < 0.f ? -(long long)mag : (long long)mag;
}
__device__ __forceinline__ long long to_fixed(double v) { return __double2ll_rn(v); }

__device__ __forceinline__ int cell_axis(int32_t packed, int a) { return (packed >> (10 * a)) & 1023; }
__device__ __forceinline__ int cell_axis(int64_t packed, int a) { return (int)((packed >> (10 * a)) & 1023); }

template <typename T> struct PointOf;
template <> struct PointOf<float> { using type = PointF; };
template <> struct PointOf<double> { using type = PointD; };

// Decompose a linear tile id into per-axis tile coordinates (axis 0 slowest).
template <int D>
__device__ __forceinline__ void tile_coords(int32_t tile, const int *ntile, int *tc) {
    int r = tile;
    for (int a = D - 1; a >= 0; --a) {
        tc[a] = r % ntile[a];
        r /= ntile[a];
    }
}

}  // namespace nfl
