// Gaussian upper tail for the FSMI pair sums, one base-2 exponential and one reciprocal on the
// SFU per evaluation.
//
//   T(s) = 0.5 * erfc(s / sqrt(log2 e)) ~= 2^(-s^2) * t * P(t),  t = 1 / (1 + p s),  s >= 0,
//
// the rational-substitution form of erfc (Hastings; Abramowitz and Stegun 7.1.26) with our own
// degree-6 coefficients, fitted for minimum absolute error of T by csrc/fit_gauss_tail.py:
// |T - exact| <= 5.1e-10 in exact arithmetic, <= 1.6e-7 (about 2 ulp of T(0) = 0.5) when
// evaluated in FP32, and <= 1e-6 T + 2e-9 everywhere. The variable s is a distance scaled by
// sqrt(log2 e) / (sigma sqrt 2), so that exp(-z^2) = 2^(-s^2).
#pragma once

#include <cuda_runtime.h>

namespace fsmi {

// p = 0.3725, fit max |T error| = 5.06e-10, FP32 max |T error| = 1.57e-07
constexpr float kTailP = 0.3725000023841858f;
constexpr float kTailC0 = 0.12908168137073517f;
constexpr float kTailC1 = 0.097091443836689f;
constexpr float kTailC2 = 0.23891545832157135f;
constexpr float kTailC3 = -0.20453312993049622f;
constexpr float kTailC4 = 0.44375884532928467f;
constexpr float kTailC5 = -0.2505171000957489f;
constexpr float kTailC6 = 0.046202804893255234f;

// sqrt(log2(e)): converts z = x / (sigma sqrt 2) into s = z sqrt(log2 e).
constexpr double kSqrtLog2e = 1.2011224087864498;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// T(|d|) for a scaled distance d >= 0 or < 0 (only |d| is used).
__device__ __forceinline__ float gauss_tail(float d)
{
    const float e = ex2_approx(-(d * d));
    const float t = rcp_approx(fmaf(kTailP, fabsf(d), 1.0f));
    float q = kTailC6;
    q = fmaf(q, t, kTailC5);
    q = fmaf(q, t, kTailC4);
    q = fmaf(q, t, kTailC3);
    q = fmaf(q, t, kTailC2);
    q = fmaf(q, t, kTailC1);
    q = fmaf(q, t, kTailC0);
    return (e * t) * q;
}

// sgn(d) T(|d|): the tail mass beyond a boundary, signed by the side it lies on.
__device__ __forceinline__ float signed_tail(float d) { return copysignf(gauss_tail(d), d); }

}  // namespace fsmi
