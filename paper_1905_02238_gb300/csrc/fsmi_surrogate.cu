// Learned surrogate of the 2D beam FSMI (not part of the paper): a 1D conv + MLP that predicts a
// beam's mutual information from its occupancy profile, trained on beams that exact FSMI labels,
// used to prescreen candidate poses before exact FSMI reranks the best of them.
//
//   input  x[256][2]: sample i of the beam at distance i + 1/2 cells; (o, 1) inside the map, (0, 0)
//          beyond it
//   conv1  2 -> 32, kernel 3, stride 2, zero padding 1, ReLU        256 -> 128 positions
//   conv2  32 -> 32, same                                           128 -> 64
//   conv3  32 -> 32, same                                           64 -> 32
//   fc1    1024 -> 256 (input index t * 32 + c), ReLU;  fc2 256 -> 1
//   conv:  z[t][c] = b[c] + sum_{k<3} sum_ci W[c][k][ci] a[2t + k - 1][ci]
//
// Parameters are one flat FP32 vector (master copy, layout below); the weights are used as a BF16
// copy of the same vector, accumulation is FP32. Training runs every layer, forward and backward,
// through one split-K SIMT GEMM whose operands are read through index functions (convolutions
// gather their im2col entries on the fly); every sum is taken in a fixed order, so a training
// step gives the same floats on every run.
#include <cuda_bf16.h>
#include <float.h>

#include "../../include/fsmi.h"
#include "fsmi_device.cuh"
#include "fsmi_internal.h"

namespace fsmi {

namespace {

constexpr int kL = 256, kCin = 2, kCh = 32, kK = 3, kHid = 256, kFlat = kCh * (kL / 8);
// flat parameter layout
constexpr int oW1 = 0, oB1 = oW1 + kCh * kK * kCin, oW2 = oB1 + kCh, oB2 = oW2 + kCh * kK * kCh, oW3 = oB2 + kCh,
              oB3 = oW3 + kCh * kK * kCh, oW4 = oB3 + kCh, oB4 = oW4 + kHid * kFlat, oW5 = oB4 + kHid,
              oB5 = oW5 + kHid, kNParams = oB5 + 1;
static_assert(kNParams == FSMI_SURR_NPARAMS, "parameter layout");

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float bf(const bf16 *p, long long i) { return __bfloat162float(p[i]); }

// ---- profiles ---------------------------------------------------------------------------------

// Sample i of a beam: the cell holding o + (i + 1/2) d, the floor of the Q31 position
// (o << 15) + (2i + 1) d (d the Q30 beam direction).
__device__ __forceinline__ void sample_2d(const float *map, int W, int H, long long ox, long long oy, int dx, int dy,
                                          int i, float &o, float &in)
{
    const long long px = ((ox << 15) + (long long)(2 * i + 1) * dx) >> 31;
    const long long py = ((oy << 15) + (long long)(2 * i + 1) * dy) >> 31;
    const bool inside = px >= 0 && px < W && py >= 0 && py < H;
    o = inside ? __ldg(map + py * W + px) : 0.0f;
    in = inside ? 1.0f : 0.0f;
}

__device__ __forceinline__ void beam_dir_2d(const int32_t *pose, const int32_t *u, int &dx, int &dy)
{
    const long long c = pose[2], s = pose[3], ux = u[0], uy = u[1];
    dx = (int)((c * ux - s * uy + (1LL << 29)) >> 30);
    dy = (int)((s * ux + c * uy + (1LL << 29)) >> 30);
}

// one warp per beam: out[n][i] = (o, inside) as BF16 pairs
__global__ void __launch_bounds__(256)
    k_profiles(const float *__restrict__ map, int W, int H, const int32_t *__restrict__ poses,
               const int32_t *__restrict__ dirs, int B, long long nbeams, const int32_t *__restrict__ beam_ids,
               long long N, __nv_bfloat162 *__restrict__ out, int *status)
{
    const int lane = lane_id();
    const long long wpb = blockDim.x >> 5;
    for (long long n = blockIdx.x * wpb + (threadIdx.x >> 5); n < N; n += (long long)gridDim.x * wpb) {
        const long long id = beam_ids ? (long long)__ldg(beam_ids + n) : n;
        if (id < 0 || id >= nbeams) {  // no such beam: an empty profile
            for (int i = lane; i < kL; i += 32) out[n * kL + i] = __floats2bfloat162_rn(0.0f, 0.0f);
            if (lane == 0) set_status(status, FSMI_STATUS_BAD_BEAM);
            continue;
        }
        const int32_t *pose = poses + 4 * (id / B);
        int dx, dy;
        beam_dir_2d(pose, dirs + 2 * (id % B), dx, dy);
        for (int i = lane; i < kL; i += 32) {
            float o, in;
            sample_2d(map, W, H, pose[0], pose[1], dx, dy, i, o, in);
            out[n * kL + i] = __floats2bfloat162_rn(o, in);
        }
    }
}

// ---- split-K SIMT GEMM with index functions ------------------------------------------------------
//
// C[m][n] = sum_k A(m, k) B(k, n); block tile 64 x 64, k-chunks of 16, 4 x 4 outputs per thread.
// With splits > 1, block z sums k in [z * kper, (z+1) * kper) and writes its partial tile to
// part[z][m][n]; k_split_reduce then adds the splits in order and applies the epilogue.

constexpr int kTM = 64, kTN = 64, kTK = 16;

template <class FA, class FB, class FE>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, int kper, FA fa, FB fb, FE fe, float *part)
{
    __shared__ float As[kTK][kTM + 4];
    __shared__ float Bs[kTK][kTN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int kbeg = blockIdx.z * kper, kend = min(K, kbeg + kper);
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += kTK) {
        for (int e = threadIdx.x; e < kTK * kTM; e += 256) {
            const int kk = e / kTM, mm = e % kTM;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < kend) ? fa(m, k) : 0.0f;
        }
        for (int e = threadIdx.x; e < kTK * kTN; e += 256) {
            const int kk = e / kTN, nn = e % kTN;
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < kend) ? fb(k, n) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m >= M || n >= N) continue;
            if (gridDim.z > 1)
                part[((size_t)blockIdx.z * M + m) * N + n] = acc[i][j];
            else
                fe(m, n, acc[i][j]);
        }
}

template <class FE>
__global__ void k_split_reduce(int M, int N, int splits, const float *__restrict__ part, FE fe)
{
    const long long MN = (long long)M * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < MN; e += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; ++z) s += part[z * MN + e];
        fe((int)(e / N), (int)(e % N), s);
    }
}

int grid_cap(long long want)
{
    const long long cap = (long long)sm_count() * 32;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

template <class FA, class FB, class FE>
cudaError_t gemm(int M, int N, int K, FA fa, FB fb, FE fe, float *part, size_t part_floats, cudaStream_t s)
{
    const int gx = (N + kTN - 1) / kTN, gy = (M + kTM - 1) / kTM;
    // split K when the output grid alone cannot fill the GPU and K is long
    int splits = 1;
    const long long blocks = (long long)gx * gy;
    while (splits < 64 && blocks * splits < 2LL * sm_count() && K / (splits * 2) >= 256 &&
           (size_t)(splits * 2) * M * N <= part_floats)
        splits *= 2;
    int kper = (K + splits - 1) / splits;
    kper = (kper + kTK - 1) / kTK * kTK;
    k_gemm<<<dim3(gx, gy, splits), 256, 0, s>>>(M, N, K, kper, fa, fb, fe, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    k_split_reduce<<<grid_cap(((long long)M * N + 255) / 256), 256, 0, s>>>(M, N, splits, part, fe);
    return cudaGetLastError();
}

// ---- training: forward -------------------------------------------------------------------------
//
// Activations (FP32, pre-ReLU) per batch of N beams: z1 [N][128][32], z2 [N][64][32],
// z3 [N][32][32], z4 [N][256]; pred, dpred [N]. Gradients of the same shapes reuse two buffers.

struct TrainBufs {
    float *z1, *z2, *z3, *z4, *pred, *dpred, *lossp, *g1, *g2, *part;
    size_t part_floats;
};

__device__ __forceinline__ float relu(float v) { return v > 0.0f ? v : 0.0f; }

// conv of layer input `in` (x as BF16 pairs for layer 1, relu(z_prev) otherwise): row m = n * Lout + t,
// column c, k-index kk = k * Cin + ci
struct ConvA1 {  // im2col of the profile (layer 1)
    const __nv_bfloat162 *x;
    __device__ float operator()(int m, int kk) const
    {
        const int n = m / 128, t = m % 128, k = kk / kCin, ci = kk % kCin;
        const int s = 2 * t + k - 1;
        if (s < 0 || s >= kL) return 0.0f;
        const __nv_bfloat162 v = x[(long long)n * kL + s];
        return ci == 0 ? __low2float(v) : __high2float(v);
    }
};
struct ConvA {  // im2col of relu(z_prev) [N][Lin][32]
    const float *z;
    int Lin;
    __device__ float operator()(int m, int kk) const
    {
        const int Lout = Lin >> 1;
        const int n = m / Lout, t = m % Lout, k = kk / kCh, ci = kk % kCh;
        const int s = 2 * t + k - 1;
        if (s < 0 || s >= Lin) return 0.0f;
        return relu(z[((long long)n * Lin + s) * kCh + ci]);
    }
};
struct WConv {  // B(kk, c) = W[c][k][ci] (BF16), kk = k * Cin + ci
    const bf16 *w;
    int cin;
    __device__ float operator()(int kk, int c) const { return bf(w, (long long)c * kK * cin + kk); }
};
struct StoreBias {  // out[m][n] = acc + b[n]
    float *out;
    const float *b;
    int ld;
    __device__ void operator()(int m, int n, float acc) const { out[(long long)m * ld + n] = acc + b[n]; }
};
struct ReluRow {  // A(m, k) = relu(z[m][k])
    const float *z;
    int ld;
    __device__ float operator()(int m, int k) const { return relu(z[(long long)m * ld + k]); }
};
struct WT {  // B(k, n) = W[n][k] (BF16 row-major [N][K])
    const bf16 *w;
    int ld;
    __device__ float operator()(int k, int n) const { return bf(w, (long long)n * ld + k); }
};

// pred[n] = b5 + sum_j W5[j] relu(z4[n][j]); lossp[n] = (pred - y)^2; dpred[n] = 2 (pred - y) / N
__global__ void k_head(const float *__restrict__ z4, const bf16 *__restrict__ w, const float *__restrict__ params,
                       const float *__restrict__ y, int N, float *pred, float *dpred, float *lossp)
{
    const int lane = lane_id();
    const int wpb = blockDim.x >> 5;
    for (int n = blockIdx.x * wpb + (threadIdx.x >> 5); n < N; n += gridDim.x * wpb) {
        float a = 0.0f;
        for (int j = lane; j < kHid; j += 32) a = fmaf(bf(w, oW5 + j), relu(z4[(long long)n * kHid + j]), a);
        a = warp_sum(a) + params[oB5];
        if (lane == 0) {
            pred[n] = a;
            if (y) {
                const float d = a - y[n];
                dpred[n] = 2.0f * d / (float)N;
                lossp[n] = d * d;
            }
        }
    }
}

// loss = sum(lossp) / N (one block, fixed order)
__global__ void __launch_bounds__(1024) k_loss(const float *__restrict__ lossp, int N, float *loss)
{
    __shared__ float sh[32];
    float a = 0.0f;
    for (int n = threadIdx.x; n < N; n += blockDim.x) a += lossp[n];
    a = warp_sum(a);
    if (lane_id() == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0f;
        v = warp_sum(v);
        if (threadIdx.x == 0) *loss = v / (float)N;
    }
}

// ---- training: backward ------------------------------------------------------------------------

// dz4[n][j] = dpred[n] W5[j] [z4 > 0]
__global__ void k_dz4(const float *__restrict__ z4, const float *__restrict__ dpred, const bf16 *__restrict__ w, int N,
                      float *__restrict__ dz4)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)N * kHid;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % kHid);
        dz4[e] = z4[e] > 0.0f ? dpred[e / kHid] * bf(w, oW5 + j) : 0.0f;
    }
}

// column sums over the batch (one block per column, fixed order): out[j] = sum_r f(r, j)
template <class F>
__global__ void __launch_bounds__(256) k_colsum(int R, int C, F f, float *out)
{
    __shared__ float sh[8];
    for (int j = blockIdx.x; j < C; j += gridDim.x) {
        float a = 0.0f;
        for (int r = threadIdx.x; r < R; r += blockDim.x) a += f(r, j);
        a = warp_sum(a);
        if (lane_id() == 0) sh[threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
            out[j] = s;
        }
        __syncthreads();
    }
}

struct Store {
    float *out;
    int ld;
    __device__ void operator()(int m, int n, float acc) const { out[(long long)m * ld + n] = acc; }
};
struct StoreMask {  // out[m][n] = acc [mask[m][n] > 0]
    float *out;
    const float *mask;
    int ld;
    __device__ void operator()(int m, int n, float acc) const
    {
        const long long i = (long long)m * ld + n;
        out[i] = mask[i] > 0.0f ? acc : 0.0f;
    }
};
struct RowT {  // A(m, k) = g[k][m] (row-major [K][ld])
    const float *g;
    int ld;
    __device__ float operator()(int m, int k) const { return g[(long long)k * ld + m]; }
};
struct RowN {  // A(m, k) = g[m][k]
    const float *g;
    int ld;
    __device__ float operator()(int m, int k) const { return g[(long long)m * ld + k]; }
};
struct WRow {  // B(k, n) = W[k][n] (BF16 row-major [K][ld])
    const bf16 *w;
    int ld;
    __device__ float operator()(int k, int n) const { return bf(w, (long long)k * ld + n); }
};
// conv weight gradient: gW[c][kk] = sum_{r = (n, t)} dz[r][c] * im2col(in)[r][kk]
struct DzT {  // A(c, r) = dz[r][c]
    const float *dz;
    __device__ float operator()(int c, int r) const { return dz[(long long)r * kCh + c]; }
};
template <class FA>
struct Im2colT {  // B(r, kk) = im2col(in)[r][kk]
    FA a;
    __device__ float operator()(int r, int kk) const { return a(r, kk); }
};
// conv data gradient: da[n][s][ci] = sum_{k, c} dz[n][t][c] W[c][k][ci], t = (s + 1 - k) / 2
struct DzGather {  // A(m = n * Lin + s, kk = k * 32 + c)
    const float *dz;
    int Lin;
    __device__ float operator()(int m, int kk) const
    {
        const int Lout = Lin >> 1;
        const int n = m / Lin, s = m % Lin, k = kk / kCh, c = kk % kCh;
        const int u = s + 1 - k;
        if (u < 0 || (u & 1)) return 0.0f;
        const int t = u >> 1;
        if (t >= Lout) return 0.0f;
        return dz[((long long)n * Lout + t) * kCh + c];
    }
};
struct WConvT {  // B(kk = k * 32 + c, ci) = W[c][k][ci]
    const bf16 *w;
    __device__ float operator()(int kk, int ci) const
    {
        const int k = kk / kCh, c = kk % kCh;
        return bf(w, ((long long)c * kK + k) * kCh + ci);
    }
};

struct SumDz {  // f(r, c) = dz[r][c]
    const float *dz;
    int ld;
    __device__ float operator()(int r, int c) const { return dz[(long long)r * ld + c]; }
};
struct W5Grad {  // f(n, j) = dpred[n] relu(z4[n][j])
    const float *dpred, *z4;
    __device__ float operator()(int n, int j) const { return dpred[n] * relu(z4[(long long)n * kHid + j]); }
};
struct B5Grad {
    const float *dpred;
    __device__ float operator()(int n, int) const { return dpred[n]; }
};

// ---- Adam --------------------------------------------------------------------------------------

// Adam (Kingma and Ba, Algorithm 1) with bias correction; also refreshes the BF16 copy.
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2, bf16 *__restrict__ wb)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        wb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_cast(const float *__restrict__ p, long long n, bf16 *__restrict__ wb)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(p[i]);
}

// ---- inference on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation) --------

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&v);
}

// Shared-memory row strides (bf16 elements) chosen so that the 8 rows one ldmatrix phase reads
// fall into 8 different 4-bank groups: 24 (48 B) for the K = 16 operands, 104 (208 B) for K = 96.
constexpr int kS1 = 24, kS2 = 104;
constexpr int kConvWarps = 4;
// per-warp buffers (bf16 elements): x [256][2]; R1 = im2col A1 [128][24] / A2 [64][104] / A3 [32][104];
// R2 = act1 [128][32] / act2 [64][32]
constexpr int kXs = kL * 2, kR1 = 64 * kS2, kR2 = 128 * kCh;
constexpr int kConvWarpElems = kXs + kR1 + kR2;
constexpr int kConvWElems = kCh * kS1 + 2 * kCh * kS2;  // W1, W2, W3

// One m16 x n32 strip of a conv layer: rows [mt * 16, mt * 16 + 16) of the im2col operand A (row
// stride sa) times W (32 rows, stride sw) over ksteps of 16; acc[nt][4] for the four n8 tiles.
__device__ __forceinline__ void conv_strip(const bf16 *A, int sa, const bf16 *Wt, int sw, int mt, int ksteps,
                                           float (&acc)[4][4])
{
    const int lane = lane_id();
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    for (int ks = 0; ks < ksteps; ++ks) {
        unsigned a0, a1, a2, a3;
        ldsm_x4(smem_u32(A + (mt * 16 + (lane & 15)) * sa + ks * 16 + 8 * (lane >> 4)), a0, a1, a2, a3);
#pragma unroll
        for (int np = 0; np < 2; ++np) {  // two n8 tiles per ldmatrix.x4
            unsigned b0, b1, b2, b3;
            const int row = np * 16 + (lane & 7) + 8 * (lane >> 4);
            ldsm_x4(smem_u32(Wt + row * sw + ks * 16 + 8 * ((lane >> 3) & 1)), b0, b1, b2, b3);
            mma_bf16(acc[2 * np], a0, a1, a2, a3, b0, b1);
            mma_bf16(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
        }
    }
}

// acc -> relu(acc + b) as bf16 pairs into act [rows][32]
__device__ __forceinline__ void store_act(bf16 *act, const float *b, int mt, const float (&acc)[4][4])
{
    const int lane = lane_id(), g = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c = nt * 8 + c2;
        const int r0 = mt * 16 + g;
        *reinterpret_cast<unsigned *>(act + r0 * kCh + c) =
            pack_bf16x2(relu(acc[nt][0] + b[c]), relu(acc[nt][1] + b[c + 1]));
        *reinterpret_cast<unsigned *>(act + (r0 + 8) * kCh + c) =
            pack_bf16x2(relu(acc[nt][2] + b[c]), relu(acc[nt][3] + b[c + 1]));
    }
}

// im2col of act [Lin][32] (stride 32) into A [Lin/2][sa]: A[t][k * 32 + ci] = act[2t + k - 1][ci]
__device__ __forceinline__ void im2col(const bf16 *act, int Lin, bf16 *A)
{
    const int Lout = Lin >> 1;
    for (int e = lane_id(); e < Lout * 3 * 4; e += 32) {  // 16-byte pieces: (t, k, quarter)
        const int q = e & 3, k = (e >> 2) % 3, t = (e >> 2) / 3;
        const int s = 2 * t + k - 1;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (s >= 0 && s < Lin) v = *reinterpret_cast<const uint4 *>(act + s * kCh + q * 8);
        *reinterpret_cast<uint4 *>(A + t * kS2 + k * kCh + q * 8) = v;
    }
}

// The conv stack of one beam: x [256][2] (bf16 pairs) in shared memory -> h0 row (1024 bf16) in
// global memory, index t * 32 + c.
__device__ void conv_stack(const __nv_bfloat162 *x, bf16 *R1, bf16 *R2, const bf16 *sW1, const bf16 *sW2,
                           const bf16 *sW3, const float *sb, bf16 *__restrict__ h0)
{
    const int lane = lane_id();
    // conv1: A1[t] = {x[2t-1], x[2t], x[2t+1], 0 x 5} as 32-bit words (k * 2 + ci order)
    for (int t = lane; t < 128; t += 32) {
        const unsigned z = 0u;
        const unsigned w0 = t > 0 ? *reinterpret_cast<const unsigned *>(x + 2 * t - 1) : z;
        const unsigned w1 = *reinterpret_cast<const unsigned *>(x + 2 * t);
        const unsigned w2 = *reinterpret_cast<const unsigned *>(x + 2 * t + 1);
        uint4 *row = reinterpret_cast<uint4 *>(R1 + t * kS1);
        row[0] = make_uint4(w0, w1, w2, z);
        row[1] = make_uint4(z, z, z, z);
    }
    __syncwarp();
    float acc[4][4];
    for (int mt = 0; mt < 8; ++mt) {
        conv_strip(R1, kS1, sW1, kS1, mt, 1, acc);
        store_act(R2, sb, mt, acc);
    }
    __syncwarp();
    im2col(R2, 128, R1);  // A2 [64][104]
    __syncwarp();
    for (int mt = 0; mt < 4; ++mt) {
        conv_strip(R1, kS2, sW2, kS2, mt, 6, acc);
        store_act(R2, sb + kCh, mt, acc);  // act2 [64][32]
    }
    __syncwarp();
    im2col(R2, 64, R1);  // A3 [32][104]
    __syncwarp();
    const int g = lane >> 2, c2 = 2 * (lane & 3);
    const float *b3 = sb + 2 * kCh;
    for (int mt = 0; mt < 2; ++mt) {
        conv_strip(R1, kS2, sW3, kS2, mt, 6, acc);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = nt * 8 + c2, t0 = mt * 16 + g;
            *reinterpret_cast<unsigned *>(h0 + t0 * kCh + c) =
                pack_bf16x2(relu(acc[nt][0] + b3[c]), relu(acc[nt][1] + b3[c + 1]));
            *reinterpret_cast<unsigned *>(h0 + (t0 + 8) * kCh + c) =
                pack_bf16x2(relu(acc[nt][2] + b3[c]), relu(acc[nt][3] + b3[c + 1]));
        }
    }
    __syncwarp();
}

// Conv stack for N beams: profiles from the map (map != nullptr; beam n = pose n / B, direction
// n % B) or given (x [N][256] bf16 pairs). h0 [N][1024] bf16.
__global__ void __launch_bounds__(kConvWarps * 32)
    k_conv_infer(const float *__restrict__ map, int W, int H, const int32_t *__restrict__ poses,
                 const int32_t *__restrict__ dirs, int B, const __nv_bfloat162 *__restrict__ xg, long long N,
                 const bf16 *__restrict__ w, const float *__restrict__ params, bf16 *__restrict__ h0,
                 unsigned long long *queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *sW1 = (bf16 *)smem_raw;
    bf16 *sW2 = sW1 + kCh * kS1;
    bf16 *sW3 = sW2 + kCh * kS2;
    float *sb = (float *)(sW3 + kCh * kS2);  // b1, b2, b3
    bf16 *wbase = (bf16 *)(sb + 3 * kCh) + (size_t)(threadIdx.x >> 5) * kConvWarpElems;
    __nv_bfloat162 *xs = (__nv_bfloat162 *)wbase;
    bf16 *R1 = wbase + kXs, *R2 = R1 + kR1;
    // weights: rows of K values, zero-padded to the row stride
    for (int e = threadIdx.x; e < kCh * kS1; e += blockDim.x) {
        const int c = e / kS1, kk = e % kS1;
        sW1[e] = kk < kK * kCin ? w[oW1 + c * kK * kCin + kk] : __float2bfloat16_rn(0.0f);
    }
    for (int e = threadIdx.x; e < kCh * kS2; e += blockDim.x) {
        const int c = e / kS2, kk = e % kS2;
        sW2[e] = kk < kK * kCh ? w[oW2 + c * kK * kCh + kk] : __float2bfloat16_rn(0.0f);
        sW3[e] = kk < kK * kCh ? w[oW3 + c * kK * kCh + kk] : __float2bfloat16_rn(0.0f);
    }
    for (int e = threadIdx.x; e < kCh; e += blockDim.x) {
        sb[e] = params[oB1 + e];
        sb[kCh + e] = params[oB2 + e];
        sb[2 * kCh + e] = params[oB3 + e];
    }
    __syncthreads();
    const int lane = lane_id();
    for_each_item(N, queue, 4, [&](long long n) {
        if (map) {
            const int32_t *pose = poses + 4 * (n / B);
            int dx, dy;
            beam_dir_2d(pose, dirs + 2 * (n % B), dx, dy);
            for (int i = lane; i < kL; i += 32) {
                float o, in;
                sample_2d(map, W, H, pose[0], pose[1], dx, dy, i, o, in);
                xs[i] = __floats2bfloat162_rn(o, in);
            }
        } else {
            for (int i = lane; i < kL; i += 32) xs[i] = xg[n * kL + i];
        }
        __syncwarp();
        conv_stack(xs, R1, R2, sW1, sW2, sW3, sb, h0 + n * kFlat);
    });
}

// fc1 + ReLU + fc2: pred[n] = b5 + sum_j W5[j] relu(b4[j] + sum_i W4[j][i] h0[n][i]).
// Block tile 128 rows x 256 columns, 16 warps (4 x 4 of 32 x 64), K in chunks of 64 through a
// double-buffered cp.async pipeline; rows of 128 B with the 16-byte chunks XOR-swizzled by row.
constexpr int kFcRows = 128, kFcK = 64, kFcThreads = 512;
constexpr int kFcStage = (kFcRows + kHid) * kFcK;  // bf16 elements per stage

__device__ __forceinline__ int swz(int row, int chunk) { return row * kFcK + ((chunk ^ (row & 7)) << 3); }

__device__ __forceinline__ void cp_async16(unsigned dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
}

__global__ void __launch_bounds__(kFcThreads)
    k_fc_infer(const bf16 *__restrict__ h0, long long N, const bf16 *__restrict__ w, const float *__restrict__ params,
               float *__restrict__ pred)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *st = (bf16 *)smem_raw;  // [2][128 + 256][64]
    float *red = (float *)(st + 2 * kFcStage);  // [128][4]
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const bf16 *W4 = w + oW4;
    for (long long r0 = (long long)blockIdx.x * kFcRows; r0 < N; r0 += (long long)gridDim.x * kFcRows) {
        auto load = [&](int stage, int kc) {
            bf16 *sa = st + stage * kFcStage, *sbm = sa + kFcRows * kFcK;
            for (int e = tid; e < (kFcRows + kHid) * 8; e += kFcThreads) {
                const int row = e >> 3, ch = e & 7;
                if (row < kFcRows) {
                    const long long gr = r0 + row;
                    const bool ok = gr < N;
                    cp_async16(smem_u32(sa + swz(row, ch)), h0 + (ok ? gr : 0) * kFlat + kc * kFcK + ch * 8, ok ? 16 : 0);
                } else {
                    const int j = row - kFcRows;
                    cp_async16(smem_u32(sbm + swz(j, ch)), W4 + (long long)j * kFlat + kc * kFcK + ch * 8, 16);
                }
            }
            asm volatile("cp.async.commit_group;");
        };
        float acc[2][8][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.0f;
        constexpr int nk = kFlat / kFcK;
        load(0, 0);
        for (int kc = 0; kc < nk; ++kc) {
            if (kc + 1 < nk) {
                load((kc + 1) & 1, kc + 1);
                asm volatile("cp.async.wait_group 1;");
            } else {
                asm volatile("cp.async.wait_group 0;");
            }
            __syncthreads();
            const bf16 *sa = st + (kc & 1) * kFcStage, *sbm = sa + kFcRows * kFcK;
#pragma unroll
            for (int ks = 0; ks < kFcK / 16; ++ks) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int row = wm * 32 + mt * 16 + (lane & 15);
                    ldsm_x4(smem_u32(sa + swz(row, ks * 2 + (lane >> 4))), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
                }
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    unsigned b0, b1, b2, b3;
                    const int row = wn * 64 + np * 16 + (lane & 7) + 8 * (lane >> 4);
                    ldsm_x4(smem_u32(sbm + swz(row, ks * 2 + ((lane >> 3) & 1))), b0, b1, b2, b3);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                        mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
                    }
                }
            }
            __syncthreads();
        }
        // epilogue: relu(acc + b4) * W5, summed over this warp's 64 columns, then over the 4 warps
        const int g = lane >> 2, c2 = 2 * (lane & 3);
        float part[2][2] = {{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = wn * 64 + nt * 8 + c2;
            const float bb0 = params[oB4 + c], bb1 = params[oB4 + c + 1];
            const float w0 = bf(w, oW5 + c), w1 = bf(w, oW5 + c + 1);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                part[mt][0] += relu(acc[mt][nt][0] + bb0) * w0 + relu(acc[mt][nt][1] + bb1) * w1;
                part[mt][1] += relu(acc[mt][nt][2] + bb0) * w0 + relu(acc[mt][nt][3] + bb1) * w1;
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v = part[mt][h];
                v += __shfl_xor_sync(kFull, v, 1);
                v += __shfl_xor_sync(kFull, v, 2);
                if ((lane & 3) == 0) red[(wm * 32 + mt * 16 + g + 8 * h) * 4 + wn] = v;
            }
        __syncthreads();
        if (tid < kFcRows && r0 + tid < N) {
            const float *rr = red + tid * 4;
            pred[r0 + tid] = params[oB5] + ((rr[0] + rr[1]) + (rr[2] + rr[3]));
        }
        __syncthreads();
    }
}

// ---- selection -------------------------------------------------------------------------------------

// Indices of the k largest of v[0..n) in descending order (ties: lower index first), by a bitonic
// sort of (value, index) keys in shared memory. One block; n <= 16384.
__global__ void __launch_bounds__(1024) k_topk(const float *__restrict__ v, int n, int k, int32_t *__restrict__ idx)
{
    extern __shared__ unsigned long long keys[];
    int m = 1;
    while (m < n) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        unsigned long long key = 0ull;  // padding sorts last
        if (i < n) {
            float f = v[i];
            if (f != f) f = -FLT_MAX;  // NaN ranks with the smallest
            unsigned u = __float_as_uint(f);
            u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // order-preserving map to unsigned
            key = ((unsigned long long)u << 32) | (unsigned)(0xFFFFFFFFu - (unsigned)i);
            if (key == 0ull) key = 1ull;
        }
        keys[i] = key;
    }
    __syncthreads();
    // descending bitonic sort
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const unsigned long long a = keys[i], b = keys[j];
                    if (desc ? (a < b) : (a > b)) {
                        keys[i] = b;
                        keys[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < k; i += blockDim.x) idx[i] = (int32_t)(0xFFFFFFFFu - (unsigned)(keys[i] & 0xFFFFFFFFull));
}

// dst[r][.] = src[idx[r]][.] for rows of `width` int32; an index outside [0, nrows) gives zeros
__global__ void k_gather_rows(const int32_t *__restrict__ src, long long nrows, int width,
                              const int32_t *__restrict__ idx, int k, int32_t *__restrict__ dst, int *status)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * width; e += gridDim.x * blockDim.x) {
        const long long r = idx[e / width];
        const bool ok = r >= 0 && r < nrows;
        if (!ok && e % width == 0) set_status(status, FSMI_STATUS_BAD_BEAM);
        dst[e] = ok ? src[r * width + e % width] : 0;
    }
}

}  // namespace

// ---- launchers -----------------------------------------------------------------------------------

size_t surrogate_train_floats(int N)
{
    const size_t n = (size_t)N;
    const size_t z = n * (128 + 64 + 32) * kCh + n * kHid;  // z1..z4
    const size_t g = n * 128 * kCh;                          // g1, g2: the largest gradient
    const size_t part = (size_t)64 * kHid * kFlat;           // split-K partials (up to 64 x the largest output)
    return z + 3 * n + 2 * g + part + 64;
}

cudaError_t launch_profiles(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                            const int32_t *beam_ids, long long N, void *out, int *status, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    k_profiles<<<grid_cap((N + 7) / 8), 256, 0, s>>>(map, W, H, poses, dirs, B, (long long)P * B, beam_ids, N,
                                                     (__nv_bfloat162 *)out, status);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_loss_grad(const float *params, const void *wbf16, const void *x, const float *y, int N,
                                       float *grad, float *loss, float *pred_out, float *ws, cudaStream_t s)
{
    const bf16 *w = (const bf16 *)wbf16;
    const __nv_bfloat162 *xb = (const __nv_bfloat162 *)x;
    TrainBufs t;
    float *q = ws;
    t.z1 = q, q += (size_t)N * 128 * kCh;
    t.z2 = q, q += (size_t)N * 64 * kCh;
    t.z3 = q, q += (size_t)N * 32 * kCh;
    t.z4 = q, q += (size_t)N * kHid;
    t.pred = q, q += N;
    t.dpred = q, q += N;
    t.lossp = q, q += N;
    t.g1 = q, q += (size_t)N * 128 * kCh;
    t.g2 = q, q += (size_t)N * 128 * kCh;
    t.part = q;
    t.part_floats = (size_t)64 * kHid * kFlat;
    cudaError_t e;
#define FSMI_TRY(x_)             \
    do {                         \
        e = (x_);                \
        if (e != cudaSuccess) return e; \
    } while (0)
    // forward
    FSMI_TRY(gemm(N * 128, kCh, kK * kCin, ConvA1{xb}, WConv{w + oW1, kCin}, StoreBias{t.z1, params + oB1, kCh},
                  t.part, t.part_floats, s));
    FSMI_TRY(gemm(N * 64, kCh, kK * kCh, ConvA{t.z1, 128}, WConv{w + oW2, kCh}, StoreBias{t.z2, params + oB2, kCh},
                  t.part, t.part_floats, s));
    FSMI_TRY(gemm(N * 32, kCh, kK * kCh, ConvA{t.z2, 64}, WConv{w + oW3, kCh}, StoreBias{t.z3, params + oB3, kCh},
                  t.part, t.part_floats, s));
    FSMI_TRY(gemm(N, kHid, kFlat, ReluRow{t.z3, kFlat}, WT{w + oW4, kFlat}, StoreBias{t.z4, params + oB4, kHid},
                  t.part, t.part_floats, s));
    float *pred = pred_out ? pred_out : t.pred;
    k_head<<<grid_cap((N + 7) / 8), 256, 0, s>>>(t.z4, w, params, y, N, pred, t.dpred, t.lossp);
    FSMI_TRY(cudaGetLastError());
    if (!y) return cudaSuccess;
    k_loss<<<1, 1024, 0, s>>>(t.lossp, N, loss);
    FSMI_TRY(cudaGetLastError());
    // backward: head
    k_colsum<<<grid_cap(kHid), 256, 0, s>>>(N, kHid, W5Grad{t.dpred, t.z4}, grad + oW5);
    k_colsum<<<1, 256, 0, s>>>(N, 1, B5Grad{t.dpred}, grad + oB5);
    float *dz4 = t.g1;  // [N][256]
    k_dz4<<<grid_cap(((long long)N * kHid + 255) / 256), 256, 0, s>>>(t.z4, t.dpred, w, N, dz4);
    FSMI_TRY(cudaGetLastError());
    k_colsum<<<grid_cap(kHid), 256, 0, s>>>(N, kHid, SumDz{dz4, kHid}, grad + oB4);
    // fc1: gW4[j][i] = sum_n dz4[n][j] relu(z3)[n][i]; dz3 = (dz4 W4) [z3 > 0]
    FSMI_TRY(gemm(kHid, kFlat, N, RowT{dz4, kHid}, ReluRow{t.z3, kFlat}, Store{grad + oW4, kFlat}, t.part,
                  t.part_floats, s));
    float *dz3 = t.g2;  // [N][32][32]
    FSMI_TRY(gemm(N, kFlat, kHid, RowN{dz4, kHid}, WRow{w + oW4, kFlat}, StoreMask{dz3, t.z3, kFlat}, t.part,
                  t.part_floats, s));
    // conv3: weights from relu(z2); data gradient into dz2 = (...) [z2 > 0]
    FSMI_TRY(gemm(kCh, kK * kCh, N * 32, DzT{dz3}, Im2colT<ConvA>{ConvA{t.z2, 64}}, Store{grad + oW3, kK * kCh},
                  t.part, t.part_floats, s));
    k_colsum<<<grid_cap(kCh), 256, 0, s>>>(N * 32, kCh, SumDz{dz3, kCh}, grad + oB3);
    float *dz2 = t.g1;  // [N][64][32]
    FSMI_TRY(gemm(N * 64, kCh, kK * kCh, DzGather{dz3, 64}, WConvT{w + oW3}, StoreMask{dz2, t.z2, kCh}, t.part,
                  t.part_floats, s));
    // conv2
    FSMI_TRY(gemm(kCh, kK * kCh, N * 64, DzT{dz2}, Im2colT<ConvA>{ConvA{t.z1, 128}}, Store{grad + oW2, kK * kCh},
                  t.part, t.part_floats, s));
    k_colsum<<<grid_cap(kCh), 256, 0, s>>>(N * 64, kCh, SumDz{dz2, kCh}, grad + oB2);
    float *dz1 = t.g2;  // [N][128][32]
    FSMI_TRY(gemm(N * 128, kCh, kK * kCh, DzGather{dz2, 128}, WConvT{w + oW2}, StoreMask{dz1, t.z1, kCh}, t.part,
                  t.part_floats, s));
    // conv1
    FSMI_TRY(gemm(kCh, kK * kCin, N * 128, DzT{dz1}, Im2colT<ConvA1>{ConvA1{xb}}, Store{grad + oW1, kK * kCin},
                  t.part, t.part_floats, s));
    k_colsum<<<grid_cap(kCh), 256, 0, s>>>(N * 128, kCh, SumDz{dz1, kCh}, grad + oB1);
#undef FSMI_TRY
    return cudaGetLastError();
}

cudaError_t launch_surrogate_adam(float *p, float *m, float *v, const float *g, float lr, float b1, float b2, float eps,
                                  int t, void *wbf16, cudaStream_t s)
{
    const float c1 = (float)(1.0 - pow((double)b1, (double)t)), c2 = (float)(1.0 - pow((double)b2, (double)t));
    k_adam<<<grid_cap((kNParams + 255) / 256), 256, 0, s>>>(p, m, v, g, kNParams, lr, b1, b2, eps, c1, c2,
                                                           (bf16 *)wbf16);
    return cudaGetLastError();
}

cudaError_t launch_surrogate_cast(const float *p, void *wbf16, cudaStream_t s)
{
    k_cast<<<grid_cap((kNParams + 255) / 256), 256, 0, s>>>(p, kNParams, (bf16 *)wbf16);
    return cudaGetLastError();
}

}  // namespace fsmi

namespace fsmi {

size_t surrogate_infer_bytes(long long N) { return kQueueBytes + (size_t)N * kFlat * sizeof(bf16); }

cudaError_t launch_surrogate_infer(const float *map, int W, int H, const int32_t *poses, const int32_t *dirs, int B,
                                   const void *x, long long N, const void *wbf16, const float *params, float *pred,
                                   void *ws, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    const bf16 *w = (const bf16 *)wbf16;
    unsigned long long *queue = (unsigned long long *)ws;
    bf16 *h0 = (bf16 *)((char *)ws + kQueueBytes);
    const size_t smem_conv = (size_t)(kConvWElems + kConvWarps * kConvWarpElems) * sizeof(bf16) + 3 * kCh * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_conv_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_conv);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_conv_infer, kConvWarps * 32, smem_conv);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sm_count() * occ;
    if (grid > (N + kConvWarps - 1) / kConvWarps) grid = (N + kConvWarps - 1) / kConvWarps;
    k_conv_infer<<<(unsigned)grid, kConvWarps * 32, smem_conv, s>>>(map, W, H, poses, dirs, B,
                                                                     (const __nv_bfloat162 *)x, N, w, params, h0, queue);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem_fc = (size_t)2 * kFcStage * sizeof(bf16) + (size_t)kFcRows * 4 * sizeof(float);
    e = cudaFuncSetAttribute(k_fc_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fc);
    if (e != cudaSuccess) return e;
    const long long tiles = (N + kFcRows - 1) / kFcRows;
    k_fc_infer<<<(unsigned)(tiles < (long long)sm_count() ? tiles : sm_count()), kFcThreads, smem_fc, s>>>(
        h0, N, w, params, pred);
    return cudaGetLastError();
}

cudaError_t launch_topk(const float *v, int n, int k, int32_t *idx, cudaStream_t s)
{
    int m = 1;
    while (m < n) m <<= 1;
    const size_t smem = (size_t)m * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(k_topk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_topk<<<1, 1024, smem, s>>>(v, n, k, idx);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const int32_t *src, long long nrows, int width, const int32_t *idx, int k,
                               int32_t *dst, int *status, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    k_gather_rows<<<grid_cap((k * width + 255) / 256), 256, 0, s>>>(src, nrows, width, idx, k, dst, status);
    return cudaGetLastError();
}

cudaError_t prepare_surrogate()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_conv_infer);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_fc_infer);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_topk);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_gather_rows);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_profiles);
    return e;
}

}  // namespace fsmi
