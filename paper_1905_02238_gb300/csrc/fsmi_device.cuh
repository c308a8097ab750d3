// Device helpers shared by the 2D and RLE kernels: warp scans, the per-cell gain, the Gaussian
// tail, integer powers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "fsmi_internal.h"

namespace fsmi {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// inclusive scans across the 32 lanes
__device__ __forceinline__ float warp_incl_add(float v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ float warp_incl_mul(float v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        float t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v *= t;
    }
    return v;
}

__device__ __forceinline__ int warp_incl_add_int(int v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Information gain of one cell whose odds are multiplied by delta (Section 2.2). Written as the
// Bernoulli KL divergence between posterior o' = o delta / (1 + a), a = o (delta - 1), and prior
// o, which equals the printed f(delta, r) and stays accurate as o -> 0 or 1:
//   f = o' log1p((delta - 1)(1 - o) / (1 + a)) - (1 - o) / (1 + a) log1p(a).
// Every operation is rounded explicitly (no contraction left to the compiler), so that the kernels
// that inline it all compute the same floats.
__device__ __forceinline__ float cell_gain(float delta, float o)
{
    const float dm1 = __fsub_rn(delta, 1.0f);
    const float a = __fmul_rn(o, dm1);
    const float ria = __fdiv_rn(1.0f, __fadd_rn(1.0f, a));
    const float omo = __fsub_rn(1.0f, o);
    const float post = __fmul_rn(__fmul_rn(o, delta), ria);
    const float l1 = log1pf(__fmul_rn(__fmul_rn(dm1, omo), ria));
    return __fsub_rn(__fmul_rn(post, l1), __fmul_rn(__fmul_rn(omo, ria), log1pf(a)));
}

// The same gain from a Chebyshev series: f(delta, o) = o (1 - o) h(o), where h is smooth on
// [0, 1] (f vanishes linearly at o = 0 and o = 1), evaluated by Clenshaw's recurrence in
// x = 2 o - 1. The host fits the series per call and keeps it only if, evaluated exactly as here,
// it stays within 1e-6 of f relative over [0, 1] (delta not too far from 1); about a third of the
// instructions of the two logarithms and the division of cell_gain.
__device__ __forceinline__ float gain_series(const float *c, float o)
{
    const float x2 = __fmaf_rn(4.0f, o, -2.0f);  // 2x
    float b1 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int k = kGainFitTerms - 1; k >= 1; --k) {
        const float b0 = __fmaf_rn(x2, b1, __fsub_rn(c[k], b2));
        b2 = b1;
        b1 = b0;
    }
    const float h = __fmaf_rn(__fmul_rn(0.5f, x2), b1, __fsub_rn(c[0], b2));
    return __fmul_rn(__fmul_rn(o, __fsub_rn(1.0f, o)), h);
}

// Upper Gaussian tail in the erfc variable: 0.5 * erfc(z) = 1 - Phi(z sqrt(2)), z >= 0.
__device__ __forceinline__ float half_erfc(float z) { return 0.5f * erfcf(z); }

// x^k for integer k >= 0 by binary powering (x^0 = 1, also for x = 0).
__device__ __forceinline__ float ipowf(float x, int k)
{
    float r = 1.0f;
    while (k > 0) {
        if (k & 1) r *= x;
        x *= x;
        k >>= 1;
    }
    return r;
}

// Chunked warp scan over the n cells held in shared memory. On entry sp = o, sc = f_occ,
// sx = f_emp. On exit sp = P(e_j), sc = C_j (sc[n] = 0), and for the uniform variant sx = D_j.
// Returns P(e_0).
__device__ __forceinline__ float cell_prefixes(float *sp, float *sc, float *sx, int n, bool want_d)
{
    const int lane = lane_id();
    const int K = ((n + 31) >> 5) | 1;  // odd block length: the lanes' blocks start in distinct banks
    const int lo = min(n, lane * K), hi = min(n, lo + K);
    float prod = 1.0f, sum = 0.0f;
    for (int i = lo; i < hi; ++i) {
        prod *= 1.0f - sp[i];
        sum += sx[i];
    }
    const float iprod = warp_incl_mul(prod);
    const float isum = warp_incl_add(sum);
    float E = __shfl_up_sync(kFull, iprod, 1);
    float q = __shfl_up_sync(kFull, isum, 1);
    if (lane == 0) {
        E = 1.0f;
        q = 0.0f;
    }
    const float pe0 = __shfl_sync(kFull, iprod, 31);
    float csum = 0.0f;
    for (int i = lo; i < hi; ++i) {
        const float o = sp[i];
        sp[i] = E * o;  // Algorithm 2
        E *= 1.0f - o;
        const float c = q + sc[i];  // Algorithm 3
        sc[i] = c;
        q += sx[i];
        csum += c;
    }
    if (want_d) {  // Algorithm 4: D_k = sum_{i<=k} C_i
        const float ic = warp_incl_add(csum);
        float Dacc = __shfl_up_sync(kFull, ic, 1);
        if (lane == 0) Dacc = 0.0f;
        for (int i = lo; i < hi; ++i) {
            Dacc += sc[i];
            sx[i] = Dacc;
        }
    }
    if (lane == 0) sc[n] = 0.0f;
    __syncwarp();
    return pe0;
}

// Warp-level work loop of the persistent evaluation kernels: calls f(item) for items 0 .. n-1,
// one warp per item. Without a queue the items are dealt out grid-stride; with one, each warp
// takes `chunk` consecutive items per atomic grab on the 64-bit counter, which must be zero at
// launch (the counter then ends at n + chunk * (number of warps)).
template <typename F>
__device__ __forceinline__ void for_each_item(long long n, unsigned long long *queue, int chunk, F &&f)
{
    const int lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    if (queue) {
        for (;;) {
            unsigned long long b0 = 0;
            if (lane == 0) b0 = atomicAdd(queue, (unsigned long long)chunk);
            b0 = __shfl_sync(kFull, b0, 0);
            if ((long long)b0 >= n) break;
            const long long b1 = min((long long)b0 + chunk, n);
            for (long long i = (long long)b0; i < b1; ++i) f(i);
        }
    } else {
        for (long long i = (long long)blockIdx.x * wpb + warp; i < n; i += (long long)gridDim.x * wpb) f(i);
    }
}

__device__ __forceinline__ void set_status(int *status, int bits)
{
    if (status) atomicOr(status, bits);
}

}  // namespace fsmi
