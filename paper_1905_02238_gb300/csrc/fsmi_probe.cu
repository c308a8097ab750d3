// Measurement kernels behind the roofline denominators of the FSMI kernels (not part of the
// method): issue rates of the SFU operations the Gaussian tail uses (ex2.approx, rcp.approx) and
// of FP32 / packed-FP32 FMAs, a streaming read (L2 bandwidth for a buffer that fits in L2, HBM for
// one that does not) and a clock spin from which the SM clock follows. The caller times each
// launch with CUDA events on the stream it passes.
#include "fsmi_internal.h"

namespace fsmi {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr float kNever = 1.2345e-38f;  // a value no probe produces: its store keeps the work alive

// Eight independent dependency chains of one operation per thread.
template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe_alu(float *sink, long long iters)
{
    float a[8];
    unsigned long long v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = 0.5f + 0.001f * (float)(threadIdx.x + i);
        asm volatile("mov.b64 %0, {%1, %1};" : "=l"(v[i]) : "f"(a[i]));
    }
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == FSMI_PROBE_EX2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[i]));
            if (OP == FSMI_PROBE_RCP) {  // the add keeps the chain away from fixed points (FMA pipe)
                asm volatile("rcp.approx.ftz.f32 %0, %0;" : "+f"(a[i]));
                asm volatile("add.f32 %0, %0, 0f3F000000;" : "+f"(a[i]));
            }
            if (OP == FSMI_PROBE_FMA) asm volatile("fma.rn.f32 %0, %0, %0, %0;" : "+f"(a[i]));
            if (OP == FSMI_PROBE_FMA2) asm volatile("fma.rn.f32x2 %0, %0, %0, %0;" : "+l"(v[i]));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float x, y;
        asm volatile("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v[i]));
        s += a[i] + x + y;
    }
    if (s == kNever) sink[0] = s;
}

// `iters` passes over n float4 of buf, each pass grid-strided, loads cached in L2 only (so that a
// thread re-reading its addresses on the next pass does not hit its own L1).
__global__ void __launch_bounds__(512) k_probe_read(const float4 *buf, long long n, long long iters, float *sink)
{
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long it = 0; it < iters; ++it) {
        long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n; i += 4 * stride) {
            const float4 x0 = __ldcg(buf + i), x1 = __ldcg(buf + i + stride);
            const float4 x2 = __ldcg(buf + i + 2 * stride), x3 = __ldcg(buf + i + 3 * stride);
            acc += (x0.x + x1.y) + (x2.z + x3.w);
        }
        for (; i < n; i += stride) acc += __ldcg(buf + i).x;
    }
    if (acc == kNever) sink[0] = acc;
}

// one warp: spin for `cycles` SM clocks (a bounded loop) and store the count
__global__ void k_probe_spin(long long cycles, long long *out)
{
    const long long c0 = clock64();
    long long c = c0;
    while (c - c0 < cycles) c = clock64();
    if (threadIdx.x == 0) *out = c - c0;
}

}  // namespace

}  // namespace fsmi

using namespace fsmi;

extern "C" fsmi_status fsmi_probe(int probe, long long iters, void *buf, size_t bytes, fsmi_stream_t stream)
{
    if (iters < 1 || !buf) return FSMI_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = sm_count();
    if (sms <= 0) return record_cuda_error(cudaGetLastError());
    switch (probe) {
        case FSMI_PROBE_EX2:
        case FSMI_PROBE_RCP:
        case FSMI_PROBE_FMA:
        case FSMI_PROBE_FMA2: {
            if (bytes < sizeof(float) || ((uintptr_t)buf & 3)) return FSMI_ERR_ARG;
            const unsigned grid = (unsigned)sms * kProbeBlocksPerSm;
            float *sink = (float *)buf;
            if (probe == FSMI_PROBE_EX2) k_probe_alu<FSMI_PROBE_EX2><<<grid, kProbeThreads, 0, s>>>(sink, iters);
            if (probe == FSMI_PROBE_RCP) k_probe_alu<FSMI_PROBE_RCP><<<grid, kProbeThreads, 0, s>>>(sink, iters);
            if (probe == FSMI_PROBE_FMA) k_probe_alu<FSMI_PROBE_FMA><<<grid, kProbeThreads, 0, s>>>(sink, iters);
            if (probe == FSMI_PROBE_FMA2) k_probe_alu<FSMI_PROBE_FMA2><<<grid, kProbeThreads, 0, s>>>(sink, iters);
            break;
        }
        case FSMI_PROBE_READ: {
            if (bytes < 16 || (bytes & 15) || ((uintptr_t)buf & 15)) return FSMI_ERR_ARG;
            k_probe_read<<<(unsigned)sms * 4, 512, 0, s>>>((const float4 *)buf, (long long)(bytes / 16), iters,
                                                            (float *)buf);
            break;
        }
        case FSMI_PROBE_SPIN: {
            if (bytes < sizeof(long long) || ((uintptr_t)buf & 7) || iters > (1LL << 40)) return FSMI_ERR_ARG;
            k_probe_spin<<<1, 32, 0, s>>>(iters, (long long *)buf);
            break;
        }
        default:
            return FSMI_ERR_ARG;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FSMI_OK : record_cuda_error(e);
}

extern "C" int fsmi_probe_threads(int probe)
{
    const int sms = sm_count();
    if (sms <= 0) return 0;
    if (probe >= FSMI_PROBE_EX2 && probe <= FSMI_PROBE_FMA2) return sms * kProbeBlocksPerSm * kProbeThreads;
    if (probe == FSMI_PROBE_READ) return sms * 4 * 512;
    if (probe == FSMI_PROBE_SPIN) return 32;
    return 0;
}
