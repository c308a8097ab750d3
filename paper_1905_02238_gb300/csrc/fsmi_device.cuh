// Device helpers shared by the 2D and RLE kernels: warp scans, the per-cell gain, the Gaussian
// tail, integer powers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

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

__device__ __forceinline__ int warp_incl_max_int(int v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane_id() >= o) v = max(v, t);
    }
    return v;
}

// Information gain of one cell whose odds are multiplied by delta (Section 2.2). Written as the
// Bernoulli KL divergence between posterior o' = o delta / (1 + a), a = o (delta - 1), and prior
// o, which equals the printed f(delta, r) and stays accurate as o -> 0 or 1:
//   f = o' log1p((delta - 1)(1 - o) / (1 + a)) - (1 - o) / (1 + a) log1p(a).
__device__ __forceinline__ float cell_gain(float delta, float o)
{
    const float dm1 = delta - 1.0f;
    const float a = o * dm1;
    const float ria = 1.0f / (1.0f + a);
    const float omo = 1.0f - o;
    const float post = o * delta * ria;
    return post * log1pf(dm1 * omo * ria) - omo * ria * log1pf(a);
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

__device__ __forceinline__ void set_status(int *status, int bits)
{
    if (status) atomicOr(status, bits);
}

}  // namespace fsmi
