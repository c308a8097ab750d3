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
// copy of the same vector, accumulation is FP32. Training keeps FP32 activations: the layers'
// products run on the tensor cores with each FP32 operand split into BF16 terms (k_gemm_tc, whose
// operands are read through index functions, convolutions gathering their im2col entries on the
// fly; k_dgrad_conv for the convolutions' data gradients), the weight and bias gradients of the
// convolutions as two-pass reductions over the batch rows (k_wgrad_part, k_colsum_part,
// k_part_final); every sum is taken in a fixed order, so a training step gives the same floats
// on every run.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched through the runtime, no -lcuda)
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <float.h>

#include <algorithm>

#include <mutex>

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
// sample i (of the first `keep`; later ones read as outside the map)
__device__ __forceinline__ void sample_2d(const float *map, int W, int H, long long ox, long long oy, int dx, int dy,
                                          int i, int keep, float &o, float &in)
{
    const long long px = ((ox << 15) + (long long)(2 * i + 1) * dx) >> 31;
    const long long py = ((oy << 15) + (long long)(2 * i + 1) * dy) >> 31;
    const bool inside = i < keep && px >= 0 && px < W && py >= 0 && py < H;
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
               const int32_t *__restrict__ dirs, int B, int keep, long long nbeams,
               const int32_t *__restrict__ beam_ids, long long N, __nv_bfloat162 *__restrict__ out, int *status)
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
            sample_2d(map, W, H, pose[0], pose[1], dx, dy, i, keep, o, in);
            out[n * kL + i] = __floats2bfloat162_rn(o, in);
        }
    }
}

// ---- split-K partial sums --------------------------------------------------------------------------
//
// The training GEMMs (k_gemm_tc, below) may split K over blocks: block z writes its partial tile to
// part[z][m][n] and k_split_reduce adds the splits in order and applies the epilogue.

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

// ---- reductions over the batch rows, in a fixed order -------------------------------------------
//
// Sums over the R rows of a batch (bias gradients, conv weight gradients) run in two passes: block
// b adds rows [b * rows, (b + 1) * rows) into part[b][...], then one thread per output adds the
// blocks' partials in block order. The row split depends only on R, so a step's gradients are the
// same floats on every run (and every GPU).
constexpr int kRedMaxBlocks = 2048;  // blocks per reduction, at most (bounds the partials)

// rows per block: at least min_rows, a multiple of 32, and few enough blocks
int red_rows(long long R, int min_rows)
{
    const long long per = (R + kRedMaxBlocks - 1) / kRedMaxBlocks;
    return (int)std::max<long long>(min_rows, (per + 31) / 32 * 32);
}

// part[b][c] = sum over the block's rows r of f(r, c), for C columns (C divides 256): the block's
// 256 / C row lanes take every (256 / C)-th row, then their sums are added in lane order. A warp
// reads consecutive columns of one row.
template <class F>
__global__ void __launch_bounds__(256) k_colsum_part(int R, int C, int rows, F f, float *__restrict__ part)
{
    __shared__ float sh[256];
    const int rl = 256 / C;
    const int c = threadIdx.x % C, rsub = threadIdx.x / C;
    const int r0 = blockIdx.x * rows, r1 = min(R, r0 + rows);
    float a = 0.0f;
    if (rsub < rl)
        for (int r = r0 + rsub; r < r1; r += rl) a += f(r, c);
    sh[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.0f;
        for (int k = 0; k < rl; ++k) t += sh[k * C + threadIdx.x];
        part[(size_t)blockIdx.x * C + threadIdx.x] = t;
    }
}

// out[o] = sum over blocks b of part[b][o], in a fixed order: a block takes 32 outputs (one per lane),
// its 8 warps the 8 contiguous eighths of the blocks, and the eighths' sums are added in order.
__global__ void __launch_bounds__(256) k_part_final(int nblk, int O, const float *__restrict__ part,
                                                    float *__restrict__ out)
{
    __shared__ float sh[8][32];
    const int lane = lane_id(), w = threadIdx.x >> 5;
    const int o = blockIdx.x * 32 + lane;
    const int b0 = (int)((long long)nblk * w / 8), b1 = (int)((long long)nblk * (w + 1) / 8);
    float t = 0.0f;
    if (o < O) {
#pragma unroll 8
        for (int b = b0; b < b1; ++b) t += part[(size_t)b * O + o];
    }
    sh[w][lane] = t;
    __syncthreads();
    if (w == 0 && o < O) {
        float u = 0.0f;
        for (int k = 0; k < 8; ++k) u += sh[k][lane];
        out[o] = u;
    }
}

// Conv weight gradient of a layer with CIN input channels, Lin input and Lout = Lin / 2 output
// positions: gW[c][k * CIN + ci] = sum over rows r = (n, t) of dz[r][c] in[n][2t + k - 1][ci], with
// `in` the layer input (relu(z) of the previous layer, or the profile x for the first). A block takes
// `rows` consecutive rows in tiles of kWgTile (Lout is a multiple of kWgTile, so a tile lies in one
// beam n, at positions t0 .. t0 + kWgTile - 1) and stages the tile's dz rows and the input positions
// 2 t0 - 1 .. 2 t0 + 2 kWgTile - 1 that its im2col rows read: row i of the tile's im2col is then the
// 3 CIN consecutive floats from offset 2 CIN i. Each thread adds its outputs over the block's rows in
// row order into part[b][...] (k_part_final adds the blocks). CIN = 32: a thread holds 4 output
// channels x 3 taps (one float4 of dz and three input values per row); CIN = 2: one output.
constexpr int kWgTile = 32;

template <int CIN>
__global__ void __launch_bounds__(256) k_wgrad_part(int R, int rows, int Lin, const float *__restrict__ dz,
                                                    const float *__restrict__ z, const __nv_bfloat162 *__restrict__ x,
                                                    float *__restrict__ part)
{
    constexpr int kNKK = kK * CIN, kO = kCh * kNKK, kPos = 2 * kWgTile + 1;
    __shared__ __align__(16) float sdz[kWgTile * kCh];
    __shared__ __align__(16) float sin_[kPos * CIN];
    const int Lout = Lin >> 1;
    const int r0 = blockIdx.x * rows, r1 = min(R, r0 + rows);
    const int tid = threadIdx.x;
    float acc[4][3] = {};
    for (int rt = r0; rt < r1; rt += kWgTile) {
        const int n = rt / Lout, t0 = rt - n * Lout;
        for (int e = tid; e < kWgTile * kCh / 4; e += 256)
            reinterpret_cast<float4 *>(sdz)[e] = reinterpret_cast<const float4 *>(dz + (long long)rt * kCh)[e];
        if (CIN == kCh) {
            for (int e = tid; e < kPos * kCh / 4; e += 256) {
                const int p = e / (kCh / 4), q = e % (kCh / 4);
                const int sidx = 2 * t0 - 1 + p;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (sidx >= 0 && sidx < Lin) {
                    v = reinterpret_cast<const float4 *>(z + ((long long)n * Lin + sidx) * kCh)[q];
                    v = make_float4(relu(v.x), relu(v.y), relu(v.z), relu(v.w));
                }
                reinterpret_cast<float4 *>(sin_)[e] = v;
            }
        } else {
            for (int p = tid; p < kPos; p += 256) {
                const int sidx = 2 * t0 - 1 + p;
                float lo = 0.0f, hi = 0.0f;
                if (sidx >= 0 && sidx < Lin) {
                    const __nv_bfloat162 v = x[(long long)n * Lin + sidx];
                    lo = __low2float(v);
                    hi = __high2float(v);
                }
                sin_[2 * p] = lo;
                sin_[2 * p + 1] = hi;
            }
        }
        __syncthreads();
        if (CIN == kCh) {
            const int cg = tid >> 5, kg = tid & 31;
            for (int i = 0; i < kWgTile; ++i) {
                const float4 d = reinterpret_cast<const float4 *>(sdz + i * kCh)[cg];
                const float *a = sin_ + 2 * CIN * i + kg;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float v = a[32 * j];
                    acc[0][j] = fmaf(d.x, v, acc[0][j]);
                    acc[1][j] = fmaf(d.y, v, acc[1][j]);
                    acc[2][j] = fmaf(d.z, v, acc[2][j]);
                    acc[3][j] = fmaf(d.w, v, acc[3][j]);
                }
            }
        } else if (tid < kO) {
            const int c = tid / kNKK, kk = tid % kNKK;
            for (int i = 0; i < kWgTile; ++i) acc[0][0] = fmaf(sdz[i * kCh + c], sin_[2 * CIN * i + kk], acc[0][0]);
        }
        __syncthreads();
    }
    float *pb = part + (size_t)blockIdx.x * kO;
    if (CIN == kCh) {
        const int cg = tid >> 5, kg = tid & 31;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) pb[(4 * cg + a) * kNKK + 32 * j + kg] = acc[a][j];
    } else if (tid < kO) {
        pb[tid] = acc[0][0];
    }
}

// out[c] = sum_r f(r, c) for C columns (C divides 256), in a fixed order (k_colsum_part, k_part_final)
template <class F>
cudaError_t colsum(int R, int C, F f, float *out, float *part, cudaStream_t s)
{
    const int rows = red_rows(R, 64), nblk = (R + rows - 1) / rows;
    k_colsum_part<<<nblk, 256, 0, s>>>(R, C, rows, f, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_part_final<<<(C + 31) / 32, 256, 0, s>>>(nblk, C, part, out);
    return cudaGetLastError();
}

// out[c * 3 CIN + k * CIN + ci] = sum over rows of dz[r][c] in[n][2t + k - 1][ci] (R = N Lout rows),
// in a fixed order (k_wgrad_part, k_part_final)
template <int CIN>
cudaError_t wgrad(int R, int Lin, const float *dz, const float *z, const __nv_bfloat162 *x, float *out, float *part,
                  cudaStream_t s)
{
    const int rows = red_rows(R, 512), nblk = (R + rows - 1) / rows;
    k_wgrad_part<CIN><<<nblk, 256, 0, s>>>(R, rows, Lin, dz, z, x, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int O = kCh * kK * CIN;
    k_part_final<<<(O + 31) / 32, 256, 0, s>>>(nblk, O, part, out);
    return cudaGetLastError();
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

__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned &r0, unsigned &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16_k8(float (&c)[4], unsigned a0, unsigned a1, unsigned b0)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a0), "r"(a1), "r"(b0));
}

// ---- training GEMMs on the tensor cores ----------------------------------------------------------
//
// C[m][n] = sum_k A(m, k) B(k, n) with FP32 operands given as index functions of (row, k), the
// products on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation). An FP32
// operand is split into BF16 terms, a_1 = bf16(a), a_2 = bf16(a - a_1), a_3 = bf16(a - a_1 - a_2),
// whose sum is a (1 + d) with |d| <= 2^-18 for two terms and 2^-27 for three (the split-BF16
// products of Henry, Tang and Heinecke, "Leveraging the bfloat16 artificial intelligence datatype
// for higher-precision computations", 2019). AS = 3 (the forward pass, whose outputs feed the loss
// and its derivative): A B = (A_1 + A_2 + A_3) B for a B of BF16 weights, exact in one term, as
// accurate as FP32 arithmetic. AS = 2 (the backward pass): A_1 B + A_2 B, plus A_1 B_2 when B is
// FP32 as well (BSPLIT; the A_2 B_2 term, below 2^-18 of the product, is left out). Block tile
// TM x TN (TM TN = 4096: 8 warps of 32 x 16 outputs, 2 x 2 MMA tiles each), K in stages of kTrK,
// staged as BF16 pairs in [row][k] order with a row pitch of kTrPitch elements (20 words: the
// fragment loads of the eight row groups fall in distinct banks). AKF / BKF: the operand's index
// function is contiguous in k (stage k-pairs across the threads) or in its row (stage rows across
// them). With more than one K split, block z writes its partial tile to part[z][m][n] and
// k_split_reduce adds the splits in order.
constexpr int kTrK = 32, kTrPitch = kTrK + 8;

// the BF16 terms of v0, v1 (t[0] = bf16(v), t[i] = bf16(v - t[0] - ... - t[i-1])) at `at` of each
// of the first `terms` arrays
__device__ __forceinline__ void split_store(bf16 *const *t, int terms, int at, float v0, float v1)
{
    for (int i = 0; i < terms; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        *reinterpret_cast<__nv_bfloat162 *>(t[i] + at) = h;
        v0 -= __low2float(h);
        v1 -= __high2float(h);
    }
}

__device__ __forceinline__ unsigned lds32(const bf16 *p) { return *reinterpret_cast<const unsigned *>(p); }

template <int TN, int AS, bool BSPLIT, bool AKF, bool BKF, class FA, class FB, class FE>
__global__ void __launch_bounds__(256) k_gemm_tc(int M, int N, int K, int kper, FA fa, FB fb, FE fe, float *part)
{
    constexpr int TM = 4096 / TN, WN = TN / 16, KP = kTrK / 2;
    static_assert(AS == 2 || AS == 3, "two or three BF16 terms of A");
    __shared__ __align__(16) bf16 sA[AS][TM * kTrPitch];
    __shared__ __align__(16) bf16 sB[BSPLIT ? 2 : 1][TN * kTrPitch];
    bf16 *const ta[3] = {sA[0], sA[1], sA[AS - 1]};
    bf16 *const tb[2] = {sB[0], sB[BSPLIT ? 1 : 0]};
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int wm = w / WN, wn = w % WN;  // the warp's outputs: rows 32 wm .., columns 16 wn ..
    const int g = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kbeg = blockIdx.z * kper, kend = min(K, kbeg + kper);
    float acc[2][2][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += kTrK) {
        for (int e = tid; e < TM * KP; e += 256) {
            const int r = AKF ? e / KP : e % TM, kp = AKF ? e % KP : e / TM;
            const int m = m0 + r, k = k0 + 2 * kp;
            float v0 = 0.0f, v1 = 0.0f;
            if (m < M) {
                if (k < kend) v0 = fa(m, k);
                if (k + 1 < kend) v1 = fa(m, k + 1);
            }
            split_store(ta, AS, r * kTrPitch + 2 * kp, v0, v1);
        }
        for (int e = tid; e < TN * KP; e += 256) {
            const int r = BKF ? e / KP : e % TN, kp = BKF ? e % KP : e / TN;
            const int n = n0 + r, k = k0 + 2 * kp;
            float v0 = 0.0f, v1 = 0.0f;
            if (n < N) {
                if (k < kend) v0 = fb(k, n);
                if (k + 1 < kend) v1 = fb(k + 1, n);
            }
            split_store(tb, BSPLIT ? 2 : 1, r * kTrPitch + 2 * kp, v0, v1);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kTrK; ks += 16) {
            unsigned a[AS][2][4], b[2][2][2];
#pragma unroll
            for (int i = 0; i < AS; ++i)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const bf16 *p = sA[i] + (32 * wm + 16 * mt + g) * kTrPitch + ks + 2 * tq;
                    a[i][mt][0] = lds32(p);
                    a[i][mt][1] = lds32(p + 8 * kTrPitch);
                    a[i][mt][2] = lds32(p + 8);
                    a[i][mt][3] = lds32(p + 8 * kTrPitch + 8);
                }
#pragma unroll
            for (int i = 0; i < (BSPLIT ? 2 : 1); ++i)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    const bf16 *p = sB[i] + (16 * wn + 8 * nt + g) * kTrPitch + ks + 2 * tq;
                    b[i][nt][0] = lds32(p);
                    b[i][nt][1] = lds32(p + 8);
                }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
                    for (int i = 0; i < AS; ++i)
                        mma_bf16(acc[mt][nt], a[i][mt][0], a[i][mt][1], a[i][mt][2], a[i][mt][3], b[0][nt][0],
                                 b[0][nt][1]);
                    if (BSPLIT)
                        mma_bf16(acc[mt][nt], a[0][mt][0], a[0][mt][1], a[0][mt][2], a[0][mt][3], b[1][nt][0],
                                 b[1][nt][1]);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + 32 * wm + 16 * mt + g + 8 * (q >> 1), n = n0 + 16 * wn + 8 * nt + 2 * tq + (q & 1);
                if (m >= M || n >= N) continue;
                if (gridDim.z > 1)
                    part[((size_t)blockIdx.z * M + m) * N + n] = acc[mt][nt][q];
                else
                    fe(m, n, acc[mt][nt][q]);
            }
}

template <int TN, int AS, bool BSPLIT, bool AKF, bool BKF, class FA, class FB, class FE>
cudaError_t gemm_tc(int M, int N, int K, FA fa, FB fb, FE fe, float *part, size_t part_floats, cudaStream_t s)
{
    constexpr int TM = 4096 / TN;
    const int gx = (N + TN - 1) / TN, gy = (M + TM - 1) / TM;
    int splits = 1;  // split K when the output grid alone cannot fill the GPU and K is long
    const long long blocks = (long long)gx * gy;
    while (splits < 64 && blocks * splits < 2LL * sm_count() && K / (splits * 2) >= 256 &&
           (size_t)(splits * 2) * M * N <= part_floats)
        splits *= 2;
    int kper = (K + splits - 1) / splits;
    kper = (kper + kTrK - 1) / kTrK * kTrK;
    k_gemm_tc<TN, AS, BSPLIT, AKF, BKF><<<dim3(gx, gy, splits), 256, 0, s>>>(M, N, K, kper, fa, fb, fe, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    k_split_reduce<<<grid_cap(((long long)M * N + 255) / 256), 256, 0, s>>>(M, N, splits, part, fe);
    return cudaGetLastError();
}

// Data gradient of a stride-2 conv layer (32 -> 32 channels) into the layer below, masked by its
// ReLU: da[n][s][ci] = [z_prev[n][s][ci] > 0] sum over the taps k and positions t with
// 2t + k - 1 = s of sum_c dz[n][t][c] W[c][k][ci]. An even s = 2u takes tap 1 at t = u, an odd
// s = 2u + 1 taps 0 at t = u + 1 and 2 at t = u (the other taps fall between positions), so a
// warp that takes the 16 positions t = u0 .. u0 + 15 of one beam (32 output positions) stages the
// dz rows u0 .. u0 + 16 (two BF16 terms each, as k_gemm_tc's backward products; row u0 + 16 is
// zero past the beam) and runs the even rows as a K = 32 product with tap 1 and the odd rows as a
// K = 64 product with taps 0 and 2: half the products of the K = 96 im2col form, whose other half
// are zeros. Weights are staged as [k][ci][c] BF16 (exact), row pitch kTrPitch.
__global__ void __launch_bounds__(256) k_dgrad_conv(int N, int Lin, const float *__restrict__ dz,
                                                    const bf16 *__restrict__ w, const float *__restrict__ zprev,
                                                    float *__restrict__ out)
{
    __shared__ __align__(16) bf16 sW[kK * kCh * kTrPitch];
    __shared__ __align__(16) bf16 sT[8][2][17 * kTrPitch];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, g = lane >> 2, tq = lane & 3;
    for (int e = tid; e < kK * kCh * kCh; e += 256) {
        const int k = e / (kCh * kCh), ci = (e / kCh) % kCh, c = e % kCh;
        sW[(k * kCh + ci) * kTrPitch + c] = w[(c * kK + k) * kCh + ci];
    }
    __syncthreads();
    const int Lout = Lin >> 1, tpb = Lout / 16;
    const long long ntiles = (long long)N * tpb;
    bf16 *const T[2] = {sT[wp][0], sT[wp][1]};
    for (long long tile = blockIdx.x * 8LL + wp; tile < ntiles; tile += gridDim.x * 8LL) {
        const int n = (int)(tile / tpb), u0 = (int)(tile % tpb) * 16;
        for (int e = lane; e < 17 * (kCh / 2); e += 32) {
            const int r = e / (kCh / 2), cp = e % (kCh / 2);
            float2 v = make_float2(0.0f, 0.0f);
            if (u0 + r < Lout) v = *reinterpret_cast<const float2 *>(dz + ((long long)n * Lout + u0 + r) * kCh + 2 * cp);
            split_store(T, 2, r * kTrPitch + 2 * cp, v.x, v.y);
        }
        __syncwarp();
        float ev[4][4] = {}, od[4][4] = {};
#pragma unroll
        for (int ks = 0; ks < kCh; ks += 16) {
            unsigned a[2][4], a1[2][4];  // rows u0 + g, + 8 (a) and u0 + g + 1, + 9 (a1)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const bf16 *p = T[i] + g * kTrPitch + ks + 2 * tq;
                a[i][0] = lds32(p);
                a[i][1] = lds32(p + 8 * kTrPitch);
                a[i][2] = lds32(p + 8);
                a[i][3] = lds32(p + 8 * kTrPitch + 8);
                a1[i][0] = lds32(p + kTrPitch);
                a1[i][1] = lds32(p + 9 * kTrPitch);
                a1[i][2] = lds32(p + kTrPitch + 8);
                a1[i][3] = lds32(p + 9 * kTrPitch + 8);
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                unsigned b[3][2];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const bf16 *q = sW + (k * kCh + nt * 8 + g) * kTrPitch + ks + 2 * tq;
                    b[k][0] = lds32(q);
                    b[k][1] = lds32(q + 8);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    mma_bf16(ev[nt], a[i][0], a[i][1], a[i][2], a[i][3], b[1][0], b[1][1]);
                    mma_bf16(od[nt], a1[i][0], a1[i][1], a1[i][2], a1[i][3], b[0][0], b[0][1]);
                    mma_bf16(od[nt], a[i][0], a[i][1], a[i][2], a[i][3], b[2][0], b[2][1]);
                }
            }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int ci = nt * 8 + 2 * tq;
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // fragment rows g, g + 8
                const int u = u0 + g + 8 * h;
#pragma unroll
                for (int odd = 0; odd < 2; ++odd) {
                    const long long i = ((long long)n * Lin + 2 * u + odd) * kCh + ci;
                    const float2 m = *reinterpret_cast<const float2 *>(zprev + i);
                    const float v0 = odd ? od[nt][2 * h] : ev[nt][2 * h], v1 = odd ? od[nt][2 * h + 1] : ev[nt][2 * h + 1];
                    *reinterpret_cast<float2 *>(out + i) = make_float2(m.x > 0.0f ? v0 : 0.0f, m.y > 0.0f ? v1 : 0.0f);
                }
            }
        }
        __syncwarp();
    }
}

cudaError_t dgrad_conv(int N, int Lin, const float *dz, const bf16 *w, const float *zprev, float *out, cudaStream_t s)
{
    const long long tiles = (long long)N * (Lin / 32);  // 16 output positions t per warp, 8 warps per block
    k_dgrad_conv<<<grid_cap((tiles + 7) / 8), 256, 0, s>>>(N, Lin, dz, w, zprev, out);
    return cudaGetLastError();
}

// Conv activations [rows][32 channels] (64 B per row) are kept in 128-byte lines of two rows;
// the 16-byte chunk (row parity, channel quarter) of line L sits at chunk ((parity << 2) | q) ^
// (L & 7). The eight rows 2t + k - 1 (t = t0 .. t0 + 7) that one ldmatrix phase reads for a conv
// tap then land in eight different bank groups, and so do the eight rows one accumulator store
// writes. Implicit GEMM: the im2col operand is addressed row by row, never materialised.
__device__ __forceinline__ int act_chunk(int r, int q)
{
    const int line = r >> 1;
    return line * 8 + ((((r & 1) << 2) | q) ^ (line & 7));  // in 16-byte units
}

constexpr int kConvWarps = 8;
constexpr int kS2 = 104;  // W2 / W3 row stride (bf16): 208 B, eight rows in eight bank groups
// per-warp buffers in 16-byte units: act1 (128 rows), then a 4 KB region that holds first the
// profile x (64 units) and conv1's operand A1 (128 rows of 16 B), later act2 (64 rows)
constexpr int kAct1Units = 128 * 4, kRegUnits = 256;
constexpr int kConvWarpUnits = kAct1Units + kRegUnits;
// block: W1 [32][8], W2 / W3 [32][104] bf16, biases, one zero chunk
constexpr int kConvWBytes = kCh * 8 * 2 + 2 * kCh * kS2 * 2 + 3 * kCh * 4 + 16;

// relu(acc + b) as bf16 pairs into a swizzled activation buffer (rows mt * 16 + g, + 8)
__device__ __forceinline__ void store_act_swz(uint4 *act, const float *b, int mt, const float (&acc)[4][4])
{
    const int lane = lane_id(), g = lane >> 2, w = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int c = nt * 8 + 2 * w;
        const int r0 = mt * 16 + g;
        unsigned *p0 = reinterpret_cast<unsigned *>(act + act_chunk(r0, nt)) + w;
        unsigned *p1 = reinterpret_cast<unsigned *>(act + act_chunk(r0 + 8, nt)) + w;
        *p0 = pack_bf16x2(relu(acc[nt][0] + b[c]), relu(acc[nt][1] + b[c + 1]));
        *p1 = pack_bf16x2(relu(acc[nt][2] + b[c]), relu(acc[nt][3] + b[c + 1]));
    }
}

// Weight fragments of a K = 96 conv layer for all 6 k-steps and 4 n8 tiles.
__device__ __forceinline__ void load_wfrag(const bf16 *Wt, unsigned (&bw)[6][4][2])
{
    const int lane = lane_id();
#pragma unroll
    for (int ks = 0; ks < 6; ++ks)
#pragma unroll
        for (int np = 0; np < 2; ++np) {
            const int row = np * 16 + (lane & 7) + 8 * (lane >> 4);
            ldsm_x4(smem_u32(Wt + row * kS2 + ks * 16 + 8 * ((lane >> 3) & 1)), bw[ks][2 * np][0], bw[ks][2 * np][1],
                    bw[ks][2 * np + 1][0], bw[ks][2 * np + 1][1]);
        }
}

// One m16 x n32 strip of a stride-2, K = 96 conv from the swizzled activations `in` (Lin rows):
// im2col row t, k-step ks (tap ks / 2, channel half ks % 2) is input row 2t + ks / 2 - 1.
__device__ __forceinline__ void conv_strip_k96(const uint4 *in, const uint4 *zero, int mt, const unsigned (&bw)[6][4][2],
                                               float (&acc)[4][4])
{
    const int lane = lane_id();
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    const int t = mt * 16 + (lane & 15);
#pragma unroll
    for (int ks = 0; ks < 6; ++ks) {
        const int r = 2 * t + (ks >> 1) - 1;
        const int q = ((ks & 1) << 1) | (lane >> 4);
        const uint4 *src = r >= 0 ? in + act_chunk(r, q) : zero;
        unsigned a0, a1, a2, a3;
        ldsm_x4(smem_u32(src), a0, a1, a2, a3);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[nt], a0, a1, a2, a3, bw[ks][nt][0], bw[ks][nt][1]);
    }
}

// The conv stack of one beam. x: profile as 256 words (bf16 pairs) in the warp's region; h0 row
// (1024 bf16, index t * 32 + c) to global memory.
__device__ void conv_stack(uint4 *act1, uint4 *reg, const uint4 *zero, const bf16 *sW1, const bf16 *sW2,
                           const bf16 *sW3, const float *sb, bf16 *__restrict__ h0)
{
    const int lane = lane_id();
    const unsigned *x = reinterpret_cast<const unsigned *>(reg);  // x[i] = (o, inside) of sample i
    uint4 *A1 = reg + 64;                                          // 128 rows x 16 B
    // conv1 operand: A1[t] = {x[2t-1], x[2t], x[2t+1], 0} (k * 2 + ci order, K padded to 8)
    for (int t = lane; t < 128; t += 32)
        A1[t] = make_uint4(t > 0 ? x[2 * t - 1] : 0u, x[2 * t], x[2 * t + 1], 0u);
    __syncwarp();
    float acc[4][4];
    {
        unsigned b[4];  // W1 fragments of the four n8 tiles (K = 8)
        ldsm_x4(smem_u32(sW1 + lane * 8), b[0], b[1], b[2], b[3]);
        for (int mt = 0; mt < 8; ++mt) {
            unsigned a0, a1;
            ldsm_x2(smem_u32(A1 + mt * 16 + (lane & 15)), a0, a1);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
                mma_bf16_k8(acc[nt], a0, a1, b[nt]);
            }
            store_act_swz(act1, sb, mt, acc);
        }
    }
    __syncwarp();
    unsigned bw[6][4][2];
    load_wfrag(sW2, bw);
    uint4 *act2 = reg;  // x and A1 are dead
    for (int mt = 0; mt < 4; ++mt) {
        conv_strip_k96(act1, zero, mt, bw, acc);
        store_act_swz(act2, sb + kCh, mt, acc);
    }
    __syncwarp();
    load_wfrag(sW3, bw);
    const int g = lane >> 2, c2 = 2 * (lane & 3);
    const float *b3 = sb + 2 * kCh;
    for (int mt = 0; mt < 2; ++mt) {
        conv_strip_k96(act2, zero, mt, bw, acc);
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
                 const int32_t *__restrict__ dirs, int B, int keep, const __nv_bfloat162 *__restrict__ xg, long long N,
                 const bf16 *__restrict__ w, const float *__restrict__ params, bf16 *__restrict__ h0,
                 unsigned long long *queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *sW1 = (bf16 *)smem_raw;        // [32][8]
    bf16 *sW2 = sW1 + kCh * 8;           // [32][104]
    bf16 *sW3 = sW2 + kCh * kS2;         // [32][104]
    float *sb = (float *)(sW3 + kCh * kS2);  // b1, b2, b3
    uint4 *zero = (uint4 *)(sb + 3 * kCh);
    uint4 *wbase = zero + 1 + (size_t)(threadIdx.x >> 5) * kConvWarpUnits;
    uint4 *act1 = wbase, *reg = wbase + kAct1Units;
    for (int e = threadIdx.x; e < kCh * 8; e += blockDim.x) {
        const int c = e / 8, kk = e % 8;
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
    if (threadIdx.x == 0) *zero = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    const int lane = lane_id();
    __nv_bfloat162 *xs = reinterpret_cast<__nv_bfloat162 *>(reg);
    for_each_item(N, queue, 4, [&](long long n) {
        if (map) {
            const int32_t *pose = poses + 4 * (n / B);
            int dx, dy;
            beam_dir_2d(pose, dirs + 2 * (n % B), dx, dy);
            for (int i = lane; i < kL; i += 32) {
                float o, in;
                sample_2d(map, W, H, pose[0], pose[1], dx, dy, i, keep, o, in);
                xs[i] = __floats2bfloat162_rn(o, in);
            }
        } else {
            for (int i = lane; i < kL; i += 32) xs[i] = xg[n * kL + i];
        }
        __syncwarp();
        conv_stack(act1, reg, zero, sW1, sW2, sW3, sb, h0 + n * kFlat);
    });
}

// ---- fc1 + ReLU + fc2 on the 5th-generation tensor cores (tcgen05, accumulators in TMEM) ------------
//
// Persistent CTAs of 6 warps, one per SM, each taking 128-row tiles: D[128][256] = h0_tile[128][1024]
// W4^T accumulates in 256 TMEM columns (FP32, row i in TMEM lane i), in one of two accumulators so
// that a tile's epilogue overlaps the next tile's MMAs. K runs in chunks of 64 through a 4-stage
// TMA pipeline; each stage holds A (128 x 64) and B (256 x 64) in the K-major layout with the
// 128-byte swizzle (16-byte chunk c of row r at c ^ (r & 7), 8-row groups 1024 B apart, 1024-byte
// aligned), written so by the tensor-map copies. Roles: warp 4 issues the copies (stage ring with
// "full" / "empty" mbarriers), warp 5 issues 4 MMAs (M = 128, N = 256, K = 16) per chunk, commits
// them to the stage's "empty" barrier and, after a tile's last chunk, to the accumulator's "tfull"
// barrier; warps 0-3 read their 32 TMEM lanes each (one row per thread), release the accumulator
// ("tempty") and form b5 + sum_j W5[j] relu(D + b4). Every wait is bounded: on timeout the kernel
// sets FSMI_STATUS_TIMEOUT, writes NaN for the rows it could not finish and returns after its
// copies and MMAs in flight have landed (again with bounded waits).

constexpr int kTcRows = 128, kTcK = 64, kTcStages = 4, kTcThreads = 192;
constexpr int kTcStageBytes = (kTcRows + kHid) * kTcK * 2;  // 48 KB
constexpr int kTcChunks = kFlat / kTcK;                      // 16
constexpr unsigned kTcAcc = 256;                             // TMEM columns per accumulator (FP32)
constexpr unsigned kTcCols = 2 * kTcAcc;
constexpr int kTcBars = 2 * kTcStages + 5;                   // full, empty, tfull[2], tempty[2], drain
constexpr size_t kTcSmem = 1024 + (size_t)kTcStages * kTcStageBytes + 8 * kTcBars + kHid * 8 + 16;
// instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1), B BF16
// (bits 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16 at bits 24-28
constexpr unsigned kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kHid >> 3) << 17) |
                              ((unsigned)(kTcRows >> 4) << 24);
constexpr long long kWaitPolls = 1LL << 22;
// poll limit of the epilogue's wait for its accumulator, per host thread (fsmi_set_wait_limit)
thread_local long long g_epi_polls = kWaitPolls;

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ unsigned long long sdesc_sw128(unsigned saddr)
{
    unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= 1ull << 16;                      // leading byte offset: not used by swizzled K-major operands
    d |= (unsigned long long)(1024 >> 4) << 32;  // stride byte offset
    d |= 1ull << 46;                      // descriptor version of the sm_100 family
    d |= 2ull << 61;                      // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned addr, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for the phase with the given parity to complete (at most `polls` tests)
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity, long long polls = kWaitPolls)
{
    for (long long i = 0; i < polls; ++i)
        if (mbar_test(addr, parity)) return true;
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                       unsigned idesc, unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(unsigned mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(unsigned taddr, float (&v)[32])
{
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void mbar_expect_tx(unsigned addr, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// TMA: a box of the 2D tensor map at (x = element along K, y = row) into shared memory, completing
// `bytes` of the mbarrier's transaction count
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap *map, int x, int y, unsigned mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned addr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ int flag_of(const int *flag) { return *(const volatile int *)flag; }

__global__ void __launch_bounds__(kTcThreads, 1)
    k_fc_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, long long N,
            const bf16 *__restrict__ w, const float *__restrict__ params, float *__restrict__ pred, int *status,
            long long epi_polls)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned long long *full = (unsigned long long *)(base + (size_t)kTcStages * kTcStageBytes);
    unsigned long long *empty = full + kTcStages;
    unsigned long long *tfull = empty + kTcStages;
    unsigned long long *tempty = tfull + 2;
    unsigned long long *drain = tempty + 2;
    float2 *bw = (float2 *)(drain + 1);  // (b4[j], W5[j])
    unsigned *tmem_slot = (unsigned *)(bw + kHid);
    __shared__ int flag;  // 0 while every wait succeeded
    const int tid = threadIdx.x, warp = tid >> 5, lane = lane_id();
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            mbar_init(smem_u32(full + i), 1);
            mbar_init(smem_u32(empty + i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(tfull + i), 1);
            mbar_init(smem_u32(tempty + i), 4);  // lane 0 of each epilogue warp
        }
        mbar_init(smem_u32(drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        flag = 0;
    }
    if (tid == 4 * 32) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmB)) : "memory");
    }
    for (int j = tid; j < kHid; j += kTcThreads) bw[j] = make_float2(params[oB4 + j], bf(w, oW5 + j));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tmem_slot;
    const long long tiles = (N + kTcRows - 1) / kTcRows;
    if (warp == 4) {
        if (lane == 0) {  // TMA producer
            long long it = 0;  // chunks issued by this CTA; stage it % S, its use number it / S
            bool ok = true;
            for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x)
                for (int kc = 0; kc < kTcChunks; ++kc) {
                    const int st = (int)(it % kTcStages);
                    const long long u = it / kTcStages;
                    if (u > 0 && !mbar_wait(smem_u32(empty + st), (unsigned)((u - 1) & 1))) ok = false;
                    if (!ok || flag_of(&flag)) {
                        ok = false;
                        break;
                    }
                    const unsigned a0 = smem_u32(base + (size_t)st * kTcStageBytes);
                    mbar_expect_tx(smem_u32(full + st), (unsigned)kTcStageBytes);
                    tma_load_2d(a0, &tmA, kc * kTcK, (int)(t * kTcRows), smem_u32(full + st));
                    tma_load_2d(a0 + kTcRows * kTcK * 2, &tmB, kc * kTcK, 0, smem_u32(full + st));
                    ++it;
                }
            // copies in flight: the last fill of every stage has landed
            for (long long j = it - 1; j >= 0 && j >= it - kTcStages; --j)
                if (!mbar_wait(smem_u32(full + (int)(j % kTcStages)), (unsigned)((j / kTcStages) & 1))) ok = false;
            if (!ok) atomicOr(&flag, 1);
        }
    } else if (warp == 5) {
        if (lane == 0) {  // MMA issuer
            long long it = 0;
            int tl = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++tl) {
                const int b = tl & 1, v = tl >> 1;
                if (v > 0 && !mbar_wait(smem_u32(tempty + b), (unsigned)((v - 1) & 1))) ok = false;
                if (!ok || flag_of(&flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned d = tmem + (unsigned)b * kTcAcc;
                for (int kc = 0; kc < kTcChunks; ++kc, ++it) {
                    const int st = (int)(it % kTcStages);
                    if (!mbar_wait(smem_u32(full + st), (unsigned)((it / kTcStages) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned a0 = smem_u32(base + (size_t)st * kTcStageBytes), b0 = a0 + kTcRows * kTcK * 2;
#pragma unroll
                    for (int k = 0; k < kTcK / 16; ++k)  // K = 16 per MMA: 32 bytes along the swizzled row
                        tc_mma(d, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), kTcIdesc, (kc | k) != 0);
                    tc_commit(smem_u32(empty + st));
                }
                if (ok) tc_commit(smem_u32(tfull + b));
            }
            if (!ok) atomicOr(&flag, 1);
            tc_commit(smem_u32(drain));  // every MMA issued has completed once this arrives
            if (!mbar_wait(smem_u32(drain), 0u)) atomicOr(&flag, 1);
        }
    } else {  // epilogue: warp w holds TMEM lanes 32w .. 32w + 31, one row per thread
        int tl = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++tl) {
            const int b = tl & 1, v = tl >> 1;
            const long long row = t * kTcRows + warp * 32 + lane;
            float acc = 0.0f;
            // the one wait whose limit the caller sets (fsmi_set_wait_limit): the producer's and the
            // MMA issuer's waits keep the full limit, so that every copy and MMA in flight has landed
            // before TMEM is freed, whatever happens here
            if (ok) ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(tfull + b), (unsigned)(v & 1), epi_polls));
            if (ok) {
                tc_fence_after();
                const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)b * kTcAcc;
                for (int c0 = 0; c0 < kHid; c0 += 32) {
                    float x[32];
                    tc_ld32(ta + (unsigned)c0, x);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float2 q = bw[c0 + j];
                        acc = fmaf(relu(x[j] + q.x), q.y, acc);
                    }
                }
                tc_fence_before();
            } else if (lane == 0) {
                atomicOr(&flag, 1);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(tempty + b));
            if (row < N) pred[row] = ok ? params[oB5] + acc : __int_as_float(0x7fc00000);
        }
    }
    __syncthreads();
    if (tid == 0 && flag != 0) set_status(status, FSMI_STATUS_TIMEOUT);
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
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
    const size_t part = (size_t)64 * kHid * kFlat;           // split-K partials (up to 64 x the largest output), also
                                                             // the batch reductions' (<= kRedMaxBlocks x 3072)
    return z + 3 * ((n + 3) & ~(size_t)3) + 2 * g + part + 64;  // pred, dpred, lossp each padded to 4 floats
}

cudaError_t launch_profiles(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                            int keep, const int32_t *beam_ids, long long N, void *out, int *status, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    k_profiles<<<grid_cap((N + 7) / 8), 256, 0, s>>>(map, W, H, poses, dirs, B, keep, (long long)P * B, beam_ids, N,
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
    auto take = [&](size_t n) {  // every buffer 16-byte aligned (float4 loads)
        float *r = q;
        q += (n + 3) & ~(size_t)3;
        return r;
    };
    t.z1 = take((size_t)N * 128 * kCh);
    t.z2 = take((size_t)N * 64 * kCh);
    t.z3 = take((size_t)N * 32 * kCh);
    t.z4 = take((size_t)N * kHid);
    t.pred = take(N);
    t.dpred = take(N);
    t.lossp = take(N);
    t.g1 = take((size_t)N * 128 * kCh);
    t.g2 = take((size_t)N * 128 * kCh);
    t.part = q;
    t.part_floats = (size_t)64 * kHid * kFlat;
    cudaError_t e;
#define FSMI_TRY(...)            \
    do {                         \
        e = (__VA_ARGS__);       \
        if (e != cudaSuccess) return e; \
    } while (0)
    // forward
    FSMI_TRY(gemm_tc<32, 3, false, true, true>(N * 128, kCh, kK * kCin, ConvA1{xb}, WConv{w + oW1, kCin},
                                            StoreBias{t.z1, params + oB1, kCh}, t.part, t.part_floats, s));
    FSMI_TRY(gemm_tc<32, 3, false, true, true>(N * 64, kCh, kK * kCh, ConvA{t.z1, 128}, WConv{w + oW2, kCh},
                                            StoreBias{t.z2, params + oB2, kCh}, t.part, t.part_floats, s));
    FSMI_TRY(gemm_tc<32, 3, false, true, true>(N * 32, kCh, kK * kCh, ConvA{t.z2, 64}, WConv{w + oW3, kCh},
                                            StoreBias{t.z3, params + oB3, kCh}, t.part, t.part_floats, s));
    FSMI_TRY(gemm_tc<64, 3, false, true, true>(N, kHid, kFlat, ReluRow{t.z3, kFlat}, WT{w + oW4, kFlat},
                                            StoreBias{t.z4, params + oB4, kHid}, t.part, t.part_floats, s));
    float *pred = pred_out ? pred_out : t.pred;
    k_head<<<grid_cap((N + 7) / 8), 256, 0, s>>>(t.z4, w, params, y, N, pred, t.dpred, t.lossp);
    FSMI_TRY(cudaGetLastError());
    if (!y) return cudaSuccess;
    k_loss<<<1, 1024, 0, s>>>(t.lossp, N, loss);
    FSMI_TRY(cudaGetLastError());
    // backward: head
    FSMI_TRY(colsum(N, kHid, W5Grad{t.dpred, t.z4}, grad + oW5, t.part, s));
    FSMI_TRY(colsum(N, 1, B5Grad{t.dpred}, grad + oB5, t.part, s));
    float *dz4 = t.g1;  // [N][256]
    k_dz4<<<grid_cap(((long long)N * kHid + 255) / 256), 256, 0, s>>>(t.z4, t.dpred, w, N, dz4);
    FSMI_TRY(cudaGetLastError());
    FSMI_TRY(colsum(N, kHid, SumDz{dz4, kHid}, grad + oB4, t.part, s));
    // fc1: gW4[j][i] = sum_n dz4[n][j] relu(z3)[n][i]; dz3 = (dz4 W4) [z3 > 0]
    FSMI_TRY(gemm_tc<64, 2, true, false, false>(kHid, kFlat, N, RowT{dz4, kHid}, ReluRow{t.z3, kFlat},
                                             Store{grad + oW4, kFlat}, t.part, t.part_floats, s));
    float *dz3 = t.g2;  // [N][32][32]
    FSMI_TRY(gemm_tc<64, 2, false, true, false>(N, kFlat, kHid, RowN{dz4, kHid}, WRow{w + oW4, kFlat},
                                             StoreMask{dz3, t.z3, kFlat}, t.part, t.part_floats, s));
    // conv3: weights from relu(z2); data gradient into dz2 = (...) [z2 > 0]
    FSMI_TRY(wgrad<kCh>(N * 32, 64, dz3, t.z2, nullptr, grad + oW3, t.part, s));
    FSMI_TRY(colsum(N * 32, kCh, SumDz{dz3, kCh}, grad + oB3, t.part, s));
    float *dz2 = t.g1;  // [N][64][32]
    FSMI_TRY(dgrad_conv(N, 64, dz3, w + oW3, t.z2, dz2, s));
    // conv2
    FSMI_TRY(wgrad<kCh>(N * 64, 128, dz2, t.z1, nullptr, grad + oW2, t.part, s));
    FSMI_TRY(colsum(N * 64, kCh, SumDz{dz2, kCh}, grad + oB2, t.part, s));
    float *dz1 = t.g2;  // [N][128][32]
    FSMI_TRY(dgrad_conv(N, 128, dz2, w + oW2, t.z1, dz1, s));
    // conv1
    FSMI_TRY(wgrad<kCin>(N * 128, kL, dz1, nullptr, xb, grad + oW1, t.part, s));
    FSMI_TRY(colsum(N * 128, kCh, SumDz{dz1, kCh}, grad + oB1, t.part, s));
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

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (looked up once)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// Row-major BF16 matrix [rows][cols] (16-byte aligned, rows of cols * 2 bytes) as a 2D tensor map
// with boxes of box_cols x box_rows and the 128-byte swizzle; out-of-range rows read as zero.
cudaError_t encode_bf16_2d(CUtensorMap *map, const void *ptr, unsigned long long cols, unsigned long long rows,
                           unsigned box_cols, unsigned box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_surrogate_infer(const float *map, int W, int H, const int32_t *poses, const int32_t *dirs, int B,
                                   int keep, const void *x, long long N, const void *wbf16, const float *params,
                                   float *pred, void *ws, int *status, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    const bf16 *w = (const bf16 *)wbf16;
    unsigned long long *queue = (unsigned long long *)ws;
    bf16 *h0 = (bf16 *)((char *)ws + kQueueBytes);
    const size_t smem_conv = (size_t)kConvWBytes + (size_t)kConvWarps * kConvWarpUnits * 16;
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
    k_conv_infer<<<(unsigned)grid, kConvWarps * 32, smem_conv, s>>>(map, W, H, poses, dirs, B, keep,
                                                                     (const __nv_bfloat162 *)x, N, w, params, h0, queue);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long tiles = (N + kTcRows - 1) / kTcRows;
    CUtensorMap tmA, tmB;
    e = encode_bf16_2d(&tmA, h0, kFlat, (unsigned long long)N, kTcK, kTcRows);
    if (e == cudaSuccess) e = encode_bf16_2d(&tmB, w + oW4, kFlat, kHid, kTcK, kHid);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fc_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    if (e != cudaSuccess) return e;
    k_fc_tc<<<(unsigned)(tiles < (long long)sm_count() ? tiles : sm_count()), kTcThreads, kTcSmem, s>>>(
        tmA, tmB, N, w, params, pred, status, g_epi_polls);
    return cudaGetLastError();
}

void set_epilogue_polls(long long polls) { g_epi_polls = polls < 0 ? kWaitPolls : polls; }

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
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_fc_tc);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_topk);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_gather_rows);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_profiles);
    return e;
}

}  // namespace fsmi
