// Issue-rate probe for the pipes the FSMI kernels lean on: ex2.approx.ftz and rcp.approx.ftz
// (SFU), fma.rn.f32 and fma.rn.f32x2 (FMA pipe), add.f32. Each thread runs eight independent
// dependency chains of one operation; 8 blocks of 256 threads per SM keep every scheduler busy.
// The SM clock is measured as well, by one warp that spins for a fixed number of clock64 cycles
// against the event-timed duration (before and after the probes), so the rates come out per SM
// per clock without assuming a clock. Prints one line per operation.
#include <cstdio>
#include <cuda_runtime.h>

enum { kEx2 = 0, kRcp = 1, kFma = 2, kFma2 = 3, kAdd = 4, kOps = 5 };

template <int OP>
__global__ void k_probe(float *out, int iters, float seed)
{
    float a[8];
    unsigned long long v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        a[i] = seed + 0.001f * (float)(threadIdx.x + i);
        asm volatile("mov.b64 %0, {%1, %1};" : "=l"(v[i]) : "f"(a[i]));
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (OP == kEx2) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[i]));
            if (OP == kRcp) {  // the add keeps the chain away from fixed points; counted as FMA-pipe work
                asm volatile("rcp.approx.ftz.f32 %0, %0;" : "+f"(a[i]));
                asm volatile("add.f32 %0, %0, 0f3F000000;" : "+f"(a[i]));
            }
            if (OP == kFma) asm volatile("fma.rn.f32 %0, %0, %0, %0;" : "+f"(a[i]));
            if (OP == kFma2) asm volatile("fma.rn.f32x2 %0, %0, %0, %0;" : "+l"(v[i]));
            if (OP == kAdd) asm volatile("add.f32 %0, %0, 0f3F000000;" : "+f"(a[i]));
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float x, y;
        asm volatile("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v[i]));
        s += a[i] + x + y;
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one warp: spin until `cycles` SM clocks have passed (a bounded loop), report the count
__global__ void k_spin(long long cycles, long long *out)
{
    const long long c0 = clock64();
    long long c = c0;
    while (c - c0 < cycles) c = clock64();
    if (threadIdx.x == 0) *out = c - c0;
}

// SM clock in MHz from one spin of about 2^24 cycles
static double sm_mhz(long long *cyc)
{
    cudaEvent_t s, e;
    cudaEventCreate(&s);
    cudaEventCreate(&e);
    float ms = 0.0f;
    long long c = 0;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(s);
        k_spin<<<1, 32>>>(1LL << 24, cyc);
        cudaEventRecord(e);
        cudaEventSynchronize(e);
        cudaEventElapsedTime(&ms, s, e);
    }
    cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost);
    cudaEventDestroy(s);
    cudaEventDestroy(e);
    return ms > 0.0f ? (double)c / (ms * 1e3) : 0.0;
}

static cudaError_t launch(int op, int blocks, int threads, float *out, int iters)
{
    switch (op) {
        case kEx2: k_probe<kEx2><<<blocks, threads>>>(out, iters, 0.5f); break;
        case kRcp: k_probe<kRcp><<<blocks, threads>>>(out, iters, 0.5f); break;
        case kFma: k_probe<kFma><<<blocks, threads>>>(out, iters, 0.5f); break;
        case kFma2: k_probe<kFma2><<<blocks, threads>>>(out, iters, 0.5f); break;
        default: k_probe<kAdd><<<blocks, threads>>>(out, iters, 0.5f); break;
    }
    return cudaGetLastError();
}

int main()
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess || sms <= 0) {
        std::fprintf(stderr, "no CUDA device\n");
        return 1;
    }
    const int blocks = sms * 8, threads = 256, iters = 4096;
    float *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(long long)) != cudaSuccess) {
        std::fprintf(stderr, "allocation failed\n");
        return 1;
    }
    cudaEvent_t s, e;
    cudaEventCreate(&s);
    cudaEventCreate(&e);
    const char *names[kOps] = {"ex2.approx.ftz.f32", "rcp.approx.ftz.f32 (+ add.f32)", "fma.rn.f32",
                               "fma.rn.f32x2 (instructions; two results each)", "add.f32"};
    const double mhz0 = sm_mhz(cyc);
    std::printf("SMs %d, %d blocks x %d threads, %d x 8 chained operations per thread; SM clock %.0f MHz\n", sms,
                blocks, threads, iters, mhz0);
    double ms_op[kOps];
    for (int op = 0; op < kOps; ++op) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {  // the first run warms up; the second is reported
            cudaEventRecord(s);
            if (launch(op, blocks, threads, out, iters) != cudaSuccess) {
                std::fprintf(stderr, "launch failed\n");
                return 1;
            }
            cudaEventRecord(e);
            cudaEventSynchronize(e);
            cudaEventElapsedTime(&ms, s, e);
        }
        ms_op[op] = ms;
    }
    const double mhz1 = sm_mhz(cyc);
    const double mhz = 0.5 * (mhz0 + mhz1);
    std::printf("SM clock after the probes %.0f MHz; rates below at the mean, %.0f MHz\n", mhz1, mhz);
    for (int op = 0; op < kOps; ++op) {
        const double lane_ops = (double)blocks * threads * iters * 8.0;
        const double per_clk = lane_ops / (ms_op[op] * 1e-3) / sms / (mhz * 1e6);
        std::printf("%-46s %8.3f ms  %7.2f lane-ops per SM per clock\n", names[op], ms_op[op], per_clk);
    }
    const cudaError_t err = cudaGetLastError();
    std::printf("status: %s\n", cudaGetErrorString(err));
    cudaFree(out);
    cudaFree(cyc);
    return err == cudaSuccess ? 0 : 1;
}
