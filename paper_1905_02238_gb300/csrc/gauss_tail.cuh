// Gaussian upper tail for the FSMI pair sums, one base-2 exponential and one reciprocal on the
// SFU per evaluation.
//
//   T(s) = 0.5 * erfc(s / sqrt(log2 e)) ~= 2^(-s^2) * t * P(t),  t = 1 / (1 + p s),  s >= 0,
//
// the rational-substitution form of erfc (Hastings; Abramowitz and Stegun 7.1.26) with our own
// degree-4 coefficients, fitted for minimum absolute error of T by csrc/fit_gauss_tail.py:
// |T - exact| <= 6.4e-8 in exact arithmetic, <= 2.3e-7 (about 4 ulp of T(0) = 0.5) when
// evaluated in FP32, and <= 3e-6 T + 5e-8 everywhere. A pair sum adds a few dozen such terms per
// cell with weights bounded by the cell's C values, so the tail contributes a few 1e-6 relative
// error to an MI at most, against the 1e-4 per-beam bar. (Degree 5 reaches 4e-9 in exact
// arithmetic but not below FP32 rounding, 1.6e-7, and costs one more packed FMA per pair of
// terms.) The variable s is a distance scaled by sqrt(log2 e) / (sigma sqrt 2), so that
// exp(-z^2) = 2^(-s^2).
#pragma once

#include <cuda_runtime.h>

namespace fsmi {

// p = 0.39, fit max |T error| = 6.31e-08, FP32 max |T error| = 2.06e-07
constexpr float kTailP = 0.38999998569488525f;
constexpr float kTailC0 = 0.12250055372714996f;
constexpr float kTailC1 = 0.2031688690185547f;
constexpr float kTailC2 = -0.08829671889543533f;
constexpr float kTailC3 = 0.3726899027824402f;
constexpr float kTailC4 = -0.11006267368793488f;

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
    float q = kTailC4;
    q = fmaf(q, t, kTailC3);
    q = fmaf(q, t, kTailC2);
    q = fmaf(q, t, kTailC1);
    q = fmaf(q, t, kTailC0);
    return (e * t) * q;
}

// ---- two tails per instruction (Blackwell packed FP32) ---------------------------------------
// Each half of an f32x2 operation is the IEEE round-to-nearest result of the scalar operation, so
// gauss_tail2 returns exactly what two gauss_tail calls return; it only halves the issue slots
// of the FP32 part.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void unpack2(f32x2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// sgn T(d0), sgn T(d1) packed, for two non-negative scaled distances packed in d; NEG (NEG1 for
// the second half, NEG by default) gives the negated tails exactly (the polynomial with negated coefficients is the negated polynomial in
// round-to-nearest arithmetic).
template <bool NEG, bool NEG1 = NEG>
__device__ __forceinline__ f32x2 gauss_tail2p(f32x2 d)
{
    constexpr float s0 = NEG ? -1.0f : 1.0f, s1 = NEG1 ? -1.0f : 1.0f;  // signs of the two halves
    float dd0, dd1, den0, den1;
    unpack2(mul2(d, d), dd0, dd1);
    const float e0 = ex2_approx(-dd0), e1 = ex2_approx(-dd1);
    unpack2(fma2(pack2(kTailP, kTailP), d, pack2(1.0f, 1.0f)), den0, den1);
    const f32x2 t = pack2(rcp_approx(den0), rcp_approx(den1));
    f32x2 q = fma2(pack2(s0 * kTailC4, s1 * kTailC4), t, pack2(s0 * kTailC3, s1 * kTailC3));
    q = fma2(q, t, pack2(s0 * kTailC2, s1 * kTailC2));
    q = fma2(q, t, pack2(s0 * kTailC1, s1 * kTailC1));
    q = fma2(q, t, pack2(s0 * kTailC0, s1 * kTailC0));
    return mul2(mul2(pack2(e0, e1), t), q);
}

// T(d0), T(d1) for two non-negative scaled distances packed in d.
__device__ __forceinline__ void gauss_tail2(f32x2 d, float &T0, float &T1)
{
    float dd0, dd1, den0, den1;
    unpack2(mul2(d, d), dd0, dd1);
    const float e0 = ex2_approx(-dd0), e1 = ex2_approx(-dd1);
    unpack2(fma2(pack2(kTailP, kTailP), d, pack2(1.0f, 1.0f)), den0, den1);
    const f32x2 t = pack2(rcp_approx(den0), rcp_approx(den1));
    f32x2 q = fma2(pack2(kTailC4, kTailC4), t, pack2(kTailC3, kTailC3));
    q = fma2(q, t, pack2(kTailC2, kTailC2));
    q = fma2(q, t, pack2(kTailC1, kTailC1));
    q = fma2(q, t, pack2(kTailC0, kTailC0));
    unpack2(mul2(mul2(pack2(e0, e1), t), q), T0, T1);
}

}  // namespace fsmi
