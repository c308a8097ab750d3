// 3D hot path (Section 4): virtual-cell sampling of each ray, run-length encoding (eq.
// occup_rle), run prefixes P_E(u), D_E(v), and the run-pair sums of FSMI-RLE (Theorem 3),
// Approx-FSMI-RLE (Theorem 5) and Uniform-FSMI-RLE (Theorem 6). One warp per ray.
//
// Run-pair terms. With x = 1 - o_u and a shift-invariant noise kernel g between virtual cells,
//   A[x, Lu, Lv, t] = sum_{j<Lu} sum_{k<Lv} x^j g(j + t - k),  B = same with weight k.
// The k-sum is a window of g: W0(m) = sum_{k<Lv} g(m - k) = Psi(m) - Psi(m - Lv) and
// W1(m) = sum_{k<Lv} k g(m - k) = m W0(m) - (Psi1(m) - Psi1(m - Lv)), with the prefix tables
// Psi(m) = sum_{d<=m} g(d), Psi1(m) = sum_{d<=m} d g(d) held in shared memory. Then
// A = sum_j x^j W0(j + t), B = sum_j x^j W1(j + t), summed only where W0 can be non-zero
// (j + t in [-K, Lv - 1 + K], K the kernel's support radius). No power x^{-t} is ever formed,
// which avoids the instability the paper notes for its alpha/beta tables (Section 4.1).
//
// Short runs. The run-pair sum is Theorem 3's regrouping of the cell-level double sum
// sum_j sum_k P(e_j) C_k g(k - j) over the virtual cells (eq. eqn_from_fsmi). When a ray's runs
// are short (mean length below kCellRunLen) that cell-level form, a banded convolution of width
// 2K + 1, costs less than the run pairs, so the ray is decompressed in shared memory and
// evaluated that way -- the switch Section 5.4 recommends between the RLE algorithm and the
// algorithm on the decompressed sequence. Both forms give the same value (pinned in the tests).
#pragma once


#include "../../include/fsmi.h"
#include "fsmi_device.cuh"
#include "gauss_tail.cuh"
#include "fsmi_internal.h"

namespace fsmi {

// Per-cell gain f(delta_occ, r) (which = 0) or f(delta_emp, r) (which = 1) of the RLE kernels: the
// host-fitted Chebyshev series when it is accurate for these deltas, else the closed form.
__device__ __forceinline__ float rle_gain(const DevParams &p, int which, float o)
{
    return p.gain_fit ? gain_series(p.gfit[which], o) : cell_gain(which ? p.demp : p.docc, o);
}

// Both gains of one o: the two series evaluated together in packed FP32 (each half of an f32x2
// operation rounds as the scalar one does, so fo and fe equal rle_gain(p, 0, o) and
// rle_gain(p, 1, o) bit for bit), or the closed forms.
__device__ __forceinline__ void rle_gains(const DevParams &p, float o, float &fo, float &fe)
{
    if (!p.gain_fit) {
        fo = cell_gain(p.docc, o);
        fe = cell_gain(p.demp, o);
        return;
    }
    const float x2 = __fmaf_rn(4.0f, o, -2.0f);  // 2x, x = 2o - 1
    const f32x2 X2 = pack2(x2, x2);
    f32x2 b1 = pack2(0.0f, 0.0f), b2 = b1;
#pragma unroll
    for (int k = kGainFitTerms - 1; k >= 1; --k) {
        const f32x2 b0 = fma2(X2, b1, sub2(pack2(p.gfit2[k][0], p.gfit2[k][1]), b2));
        b2 = b1;
        b1 = b0;
    }
    const f32x2 h = fma2(mul2(pack2(0.5f, 0.5f), X2), b1, sub2(pack2(p.gfit2[0][0], p.gfit2[0][1]), b2));
    const float w = __fmul_rn(o, __fsub_rn(1.0f, o));
    unpack2(mul2(pack2(w, w), h), fo, fe);
}

// ---- noise-kernel prefix tables --------------------------------------------------------------

// tab[i] = (Psi(m), Psi1(m)) for m = i - K - 1, i in [0, 2K + 1]; Psi(-K-1) = 0, Psi(K) = total;
// gtab[K + d] = g(d). The host builds both once per launch (fill_rle_table: kind 0 Gaussian
// density (Theorem 3), 1 Gaussian cell mass, 2 box 1[|d| <= H] (Theorem 6); band >= 0 zeroes
// |d| > band, the strict-band reading of Approx-FSMI-RLE; normalisation folded into g; in double,
// stored as float); each block copies them from the launch's parameters into shared memory.
static __device__ void load_table(float2 *tab, float *gtab, int K, const RleTable &t)
{
    for (int i = threadIdx.x; i < 2 * K + 2; i += blockDim.x) tab[i] = t.tab[i];
    for (int i = threadIdx.x; i < 2 * K + 1; i += blockDim.x) gtab[i] = t.gtab[i];
    __syncthreads();
}

__device__ __forceinline__ float2 tab_at(const float2 *tab, int K, int m)
{
    return tab[min(max(m, -K - 1), K) + K + 1];
}

// A and B of one run pair (see the file comment).
__device__ __forceinline__ void pair_AB(float x, int Lu, int Lv, int t, const float2 *tab, int K, float &A,
                                        float &B)
{
    A = 0.0f;
    B = 0.0f;
    const int jlo = max(0, -K - t);
    const int jhi = min(Lu - 1, Lv - 1 + K - t);
    if (jlo > jhi) return;
    float xp = ipowf(x, jlo);
    for (int j = jlo; j <= jhi; ++j) {
        const int m = j + t;
        const float2 a = tab_at(tab, K, m);
        const float2 b = tab_at(tab, K, m - Lv);
        const float w0 = a.x - b.x;
        const float w1 = fmaf((float)m, w0, -(a.y - b.y));
        A = fmaf(xp, w0, A);
        B = fmaf(xp, w1, B);
        xp *= x;
    }
}

// ---- per-ray run arrays in shared memory ----------------------------------------------------

struct RunSmem {
    float *O;  // o_u, then P_E(u) o_u
    float *X;  // 1 - o_u
    float *A;  // D_E(u) + f(delta_occ, r_u)
    float *F;  // f(delta_emp, r_u)
    int *S;    // s_u (first virtual cell of run u); S[nr] = n
    int *L;    // L_u
};

__device__ __forceinline__ RunSmem run_smem(float *base, int stride)
{
    RunSmem r;
    r.O = base;
    r.X = base + stride;
    r.A = base + 2 * stride;
    r.F = base + 3 * stride;
    r.S = (int *)(base + 4 * stride);
    r.L = (int *)(base + 5 * stride);
    return r;
}

// Run starts s_u = sum_{i<u} L_i (and S[nr] = n) from the lengths, or lengths from the starts.
static __device__ void run_starts(const RunSmem &r, int nr, bool have_s)
{
    const int lane = lane_id();
    const int K = (nr + 31) >> 5;
    const int lo = min(nr, lane * K), hi = min(nr, lo + K);
    if (!have_s) {
        int cs = 0;
        for (int u = lo; u < hi; ++u) cs += r.L[u];
        const int ic = warp_incl_add_int(cs);
        int s = __shfl_up_sync(kFull, ic, 1);
        if (lane == 0) s = 0;
        for (int u = lo; u < hi; ++u) {
            r.S[u] = s;
            s += r.L[u];
        }
        if (lane == 31) r.S[nr] = ic;
    } else {
        for (int u = lo; u < hi; ++u) r.L[u] = r.S[u + 1] - r.S[u];
    }
    __syncwarp();
}

// Run prefixes (Algorithms for P_E(u) and D_E(v)): P_E(u) = prod_{i<u} (1 - o_i)^{L_i},
// D_E(u) = sum_{i<u} L_i f(delta_emp, r_i). On entry O, L and S are set.
static __device__ void run_prefixes(const RunSmem &r, int nr, const DevParams &p)
{
    const int lane = lane_id();
    const int K = (nr + 31) >> 5;
    const int lo = min(nr, lane * K), hi = min(nr, lo + K);
    float prod = 1.0f, sum = 0.0f;
    for (int u = lo; u < hi; ++u) {
        const float o = r.O[u];
        const int L = r.L[u];
        prod *= ipowf(1.0f - o, L);
        sum = fmaf((float)L, rle_gain(p, 1, o), sum);
    }
    const float ip = warp_incl_mul(prod);
    const float is = warp_incl_add(sum);
    float E = __shfl_up_sync(kFull, ip, 1);
    float D = __shfl_up_sync(kFull, is, 1);
    if (lane == 0) {
        E = 1.0f;
        D = 0.0f;
    }
    for (int u = lo; u < hi; ++u) {
        const float o = r.O[u];
        const int L = r.L[u];
        const float x = 1.0f - o;
        const float fe = rle_gain(p, 1, o);
        r.X[u] = x;
        r.F[u] = fe;
        r.A[u] = D + rle_gain(p, 0, o);
        r.O[u] = E * o;
        E *= ipowf(x, L);
        D = fmaf((float)L, fe, D);
    }
    __syncwarp();
}

// Eq. (group_fsmi_rle_exact) over every run pair whose A, B can be non-zero (FSMI-RLE,
// Uniform-FSMI-RLE, strict-band Approx-FSMI-RLE); returns this lane's partial sum.
static __device__ float pairs_all(const RunSmem &r, int nr, const float2 *tab, int K)
{
    float tot = 0.0f;
    for (int u = lane_id(); u < nr; u += 32) {
        const float Pu = r.O[u];
        if (Pu == 0.0f) continue;
        const float x = r.X[u];
        const int su = r.S[u], Lu = r.L[u];
        float acc = 0.0f;
        for (int v = 0; v < nr; ++v) {
            const int t = su - r.S[v];
            const int Lv = r.L[v];
            if (t + Lu - 1 < -K || t > Lv - 1 + K) continue;
            float A, B;
            pair_AB(x, Lu, Lv, t, tab, K, A, B);
            acc = fmaf(r.A[v], A, fmaf(r.F[v], B, acc));
        }
        tot = fmaf(Pu, acc, tot);
    }
    return tot;
}

// Theorem 5 as printed: the full diagonal block (theta, gamma) plus, for runs within Delta of
// each other, the sub-blocks s', L' of eqs. (su')-(Lv') with shift t = s_u' - s_v', weighted by
// (1 - o_u)^{s_u' - s_u} (u < v) or with D_E(v) + (s_v' - s_v) f(delta_emp, r_v) (u > v).
static __device__ float pairs_thm5(const RunSmem &r, int nr, const float2 *tab, int K, int D)
{
    float tot = 0.0f;
    for (int u = lane_id(); u < nr; u += 32) {
        const float Pu = r.O[u];
        if (Pu == 0.0f) continue;
        const float x = r.X[u];
        const int su = r.S[u], Lu = r.L[u];
        float A, B;
        pair_AB(x, Lu, Lu, 0, tab, K, A, B);
        float acc = fmaf(r.A[u], A, r.F[u] * B);
        for (int v = u + 1; v < nr; ++v) {
            const int sv = r.S[v];
            if (!(sv < su + Lu + D)) break;
            const int Lv = r.L[v];
            const int su2 = max(su, sv - D);
            const int Lu2 = su + Lu - su2;
            const int Lv2 = min(Lv, su + Lu + D - sv);
            pair_AB(x, Lu2, Lv2, su2 - sv, tab, K, A, B);
            acc = fmaf(ipowf(x, su2 - su), fmaf(r.A[v], A, r.F[v] * B), acc);
        }
        for (int v = u - 1; v >= 0; --v) {
            const int sv = r.S[v], Lv = r.L[v];
            if (!(su < sv + Lv + D)) break;
            const int Lu2 = min(Lu, sv + Lv + D - su);
            const int sv2 = max(sv, su - D);
            const int Lv2 = sv + Lv - sv2;
            pair_AB(x, Lu2, Lv2, su - sv2, tab, K, A, B);
            acc = fmaf(fmaf((float)(sv2 - sv), r.F[v], r.A[v]), A, fmaf(r.F[v], B, acc));
        }
        tot = fmaf(Pu, acc, tot);
    }
    return tot;
}

constexpr int kArraysRLE = 7;                  // per-warp shared arrays (each `stride` floats)

// run containing virtual cell i: the last u with S[u] <= i
__device__ __forceinline__ int run_of(const int *S, int nr, int i)
{
    int lo = 0, len = nr;
    while (len > 0) {
        const int half = len >> 1;
        if (S[lo + half] <= i) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo - 1;
}

// sum_j P(e_j) sum_{|d| <= K} g(d) C_{j+d} over j in this lane's cells (P in CP, C at CC[K + k],
// zero-padded by K on both sides), the taps added in increasing d. A compile-time radius KK keeps
// the 2 KK + 1 kernel values in registers for the whole ray (one shared load per tap instead of
// two); both forms add the same products in the same order. Only the kernels of the other
// variants take this register form (FIXED); the Theorem 5 kernel, whose rays mostly take its
// windowed cell form, keeps the taps in registers in window_conv_k instead.
template <int KK>
__device__ __forceinline__ float band_conv_k(const float *CP, const float *CC, const float *gtab, int n)
{
    float g[2 * KK + 1];
#pragma unroll
    for (int d = 0; d <= 2 * KK; ++d) g[d] = gtab[d];
    float v = 0.0f;
    for (int j = lane_id(); j < n; j += 32) {
        float acc = 0.0f;
#pragma unroll
        for (int d = 0; d <= 2 * KK; ++d) acc = fmaf(g[d], CC[j + d], acc);
        v = fmaf(CP[j], acc, v);
    }
    return v;
}

template <bool FIXED>
__device__ __forceinline__ float band_conv(const float *CP, const float *CC, const float *gtab, int K, int n)
{
    if (FIXED && K == 15) return band_conv_k<15>(CP, CC, gtab, n);  // Gaussian kernels at sigma = 2 cells
    if (FIXED && K == 6) return band_conv_k<6>(CP, CC, gtab, n);    // strict band, Delta = 6
    if (FIXED && K == 4) return band_conv_k<4>(CP, CC, gtab, n);    // box kernel, H = 4
    float v = 0.0f;
    for (int j = lane_id(); j < n; j += 32) {
        float acc = 0.0f;
        for (int d = -K; d <= K; ++d) acc = fmaf(gtab[K + d], CC[K + j + d], acc);
        v = fmaf(CP[j], acc, v);
    }
    return v;
}

// Theorem 5 at the cell level. The pairs (j, k) its sub-blocks keep (the whole diagonal block of
// each run, and for runs u < v the cells j >= s_v - Delta of run u with the cells k < e_u + Delta
// of run v, and the mirror image) are, for a first-hit cell j of run u, the contiguous cells
// [lo_j, hi_j) with lo_j = max(s of the run holding j - Delta, s_u - Delta) and
// hi_j = min(e_u + Delta, e of the run holding j + Delta) (cells clamped to [0, n); s, e a run's
// first cell and one past its last). So Theorem 5 is sum_j P(e_j) sum_{k in [lo_j, hi_j)} g(k - j)
// C_k, taken here with the taps |k - j| <= K of the banded convolution, in increasing k. RI holds
// each cell's run index, S the run starts (S[nr] = n).
__device__ __forceinline__ float window_conv(const float *CP, const float *CC, const float *gtab, int K, int n,
                                             const int *S, const int *RI, int D)
{
    float v = 0.0f;
    for (int j = lane_id(); j < n; j += 32) {
        const int u = RI[j];
        const int a = max(j - D, 0), b = min(j + D, n - 1);
        const int lo = max(S[RI[a]], S[u] - D), hi = min(S[u + 1] + D, S[RI[b] + 1]);
        const int d0 = max(lo - j, -K), d1 = min(hi - j, K + 1);
        float acc = 0.0f;
        for (int d = d0; d < d1; ++d) acc = fmaf(gtab[K + d], CC[K + j + d], acc);
        v = fmaf(CP[j], acc, v);
    }
    return v;
}

// window_conv with a compile-time radius KK: the 2 KK + 1 kernel values in registers and every tap
// predicated on the window, so that no lane waits for another's longer window; the same products
// added in the same order (bit-identical).
template <int KK>
__device__ __forceinline__ float window_conv_k(const float *CP, const float *CC, const float *gtab, int n, const int *S,
                                               const int *RI, int D)
{
    float g[2 * KK + 1];
#pragma unroll
    for (int d = 0; d <= 2 * KK; ++d) g[d] = gtab[d];
    float v = 0.0f;
    for (int j = lane_id(); j < n; j += 32) {
        const int u = RI[j];
        const int a = max(j - D, 0), b = min(j + D, n - 1);
        const int lo = max(S[RI[a]], S[u] - D), hi = min(S[u + 1] + D, S[RI[b] + 1]);
        const int d0 = lo - j + KK, w = hi - lo;  // taps d0 .. d0 + w - 1 of 0 .. 2 KK
        float acc = 0.0f;
#pragma unroll
        for (int d = 0; d <= 2 * KK; ++d)
            if ((unsigned)(d - d0) < (unsigned)w) acc = fmaf(g[d], CC[j + d], acc);
        v = fmaf(CP[j], acc, v);
    }
    return v;
}

// Cell-level evaluation (eq. eqn_from_fsmi) of one ray: decompress the runs into the n virtual
// cells, form P(e_j) and C_k by warp scans (Algorithms 2 and 3), then
// I = sum_j P(e_j) sum_{|d| <= K} g(d) C_{j+d} (FSMI-RLE, Uniform-FSMI-RLE, strict-band
// Approx-FSMI-RLE), or for Theorem 5 the same sum over each first-hit cell's window of kept pairs
// (window_conv). Arrays: 0 run o, 1 run f_occ (then, for Theorem 5, each cell's run index), 2 run
// f_emp, 3 P, 4 run starts S, 5 f_emp per cell, 6 C padded by K zeros on both sides.
static __device__ float ray_mi_cells(float *base, int stride, int nr, int n, const DevParams &p, const float *gtab, int K,
                                     bool thm5)
{
    const int lane = lane_id();
    float *O = base, *RFO = base + stride, *RFE = base + 2 * stride, *CP = base + 3 * stride;
    const int *S = (const int *)(base + 4 * stride);
    float *CF = base + 5 * stride, *CC = base + 6 * stride;
    for (int u = lane; u < nr; u += 32) {
        float fo, fe;
        rle_gains(p, O[u], fo, fe);
        RFO[u] = fo;
        RFE[u] = fe;
    }
    for (int i = lane; i < K; i += 32) {
        CC[i] = 0.0f;
        CC[K + n + i] = 0.0f;
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        const int u = run_of(S, nr, i);
        CP[i] = O[u];
        CC[K + i] = RFO[u];
        CF[i] = RFE[u];
    }
    __syncwarp();
    cell_prefixes(CP, CC + K, CF, n, false);  // CP = P(e_j), CC[K + k] = C_k, CC[K + n] = 0
    if (thm5) {
        int *RI = (int *)RFO;  // the run gains are spread to the cells by now
        for (int i = lane; i < n; i += 32) RI[i] = run_of(S, nr, i);
        __syncwarp();
        return window_conv(CP, CC, gtab, K, n, S, RI, p.trunc);
    }
    return band_conv<false>(CP, CC, gtab, K, n);
}

__device__ __forceinline__ float ray_mi(float *base, int stride, int nr, const DevParams &p, const float2 *tab,
                                        const float *gtab, int K, bool have_s)
{
    if (nr <= 0) return 0.0f;
    const RunSmem r = run_smem(base, stride);
    run_starts(r, nr, have_s);
    const int n = r.S[nr];
    const bool thm5 = p.variant == FSMI_APPROX && p.approx_reading == 0;
    float v;
    if (n < p.cell_runlen * nr) {
        v = ray_mi_cells(base, stride, nr, n, p, gtab, K, thm5);
    } else {
        run_prefixes(r, nr, p);
        if (p.variant == FSMI_APPROX && p.approx_reading == 0)
            v = pairs_thm5(r, nr, tab, K, p.trunc);
        else
            v = pairs_all(r, nr, tab, K);
    }
    return warp_sum(v);
}

// ---- sampling and encoding -------------------------------------------------------------------

// Virtual cells of ray `ray` (= pose * R + r): sample i is the voxel holding
// o + (i + 1/2) d, i.e. floor of the Q31 position (o << 15) + (2i + 1) d, for i < nsamp until the
// first sample outside the grid. Runs are maximal spans of bit-identical values split every `cap`
// cells from the span's start. Writes O[u] = value, S[u] = first cell, S[nr] = n; returns nr.
//
// Fused form (CP != nullptr): also writes every virtual cell's o (CP) and, in SP[k], the value of
// the k-th span of equal values (k counted over the ray; *nspan_out receives their number), from
// which span_gains fills in the cells' gains; with RI, every cell's run index. Runs past nrcap are
// counted but not stored; *n_out receives n.
static __device__ int sample_encode_ray(const float *__restrict__ vox, int X, int Y, int Z, const int32_t *pose,
                                        const int32_t *u, int nsamp, int cap, float *O, int *S, int nrcap, int *n_out,
                                        float *CP, float *SP, int *nspan_out, int *RI = nullptr)
{
    const int lane = lane_id();
    int nspan = 0;
    long long d[3], o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const long long acc = (long long)pose[3 + 3 * a] * u[0] + (long long)pose[4 + 3 * a] * u[1] +
                              (long long)pose[5 + 3 * a] * u[2];
        d[a] = (acc + (1LL << 29)) >> 30;
        o[a] = (long long)pose[a] << 15;
    }
    int nrun = 0, carried = 0, n = 0;
    unsigned prev_bits = 0u;
    // Q31 position o + (2i + 1) d of this lane's sample, advanced by 64 d per chunk of 32
    long long q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) q[a] = o[a] + (2LL * lane + 1) * d[a];
    const float inv_cap = 1.0f / (float)cap;
    const unsigned lane_le = 0xffffffffu >> (31 - lane);  // lanes 0 .. lane
    // this lane's sample of the chunk at `base`: whether it lies in the grid, and its voxel value
    auto fetch = [&](int i, bool &inb, float &val) {
        inb = false;
        val = 0.0f;
        if (i < nsamp) {
            // voxel = position >> 31; positions stay far below 2^62, so the low 32 bits of the
            // shifted value are the voxel when it is in the grid and a value >= the extent (as
            // unsigned) when it is not, negative positions included
            const unsigned px = (unsigned)(q[0] >> 31), py = (unsigned)(q[1] >> 31), pz = (unsigned)(q[2] >> 31);
            inb = px < (unsigned)X && py < (unsigned)Y && pz < (unsigned)Z;
            if (inb) val = __ldg(vox + ((size_t)(pz * (unsigned)Y + py) * (unsigned)X + px));
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) q[a] += 64 * d[a];
    };
    // the next chunk's gathers are issued before the current chunk is encoded
    bool inb_next;
    float val_next;
    fetch(lane, inb_next, val_next);
    for (int base = 0; base < nsamp; base += 32) {
        const int i = base + lane;
        const bool inb = inb_next;
        const float val = val_next;
        if (__all_sync(kFull, inb)) fetch(i + 32, inb_next, val_next);  // a chunk with a sample outside is the last
        const unsigned m_in = __ballot_sync(kFull, inb);
        const int nvalid = (m_in == kFull) ? 32 : (__ffs(~m_in) - 1);
        const bool valid = lane < nvalid;
        const unsigned bits = __float_as_uint(val);
        unsigned pbits = __shfl_up_sync(kFull, bits, 1);
        if (lane == 0) pbits = prev_bits;
        const bool newval = valid && (i == 0 || bits != pbits);
        // start of this cell's span of equal values: the last lane at or before this one where a new
        // value begins, else the span carried over from the previous chunk
        const unsigned mnew = __ballot_sync(kFull, newval);
        const unsigned nle = mnew & lane_le;
        const int st = nle ? base + 31 - __clz(nle) : carried;
        // a run of equal values splits every cap samples: (i - st) a multiple of cap, found with a
        // rounded quotient (exact: i - st < 2^20 and cap <= 255) instead of an integer remainder
        const int rel = i - st;
        const bool brk = valid && rel - __float2int_rn((float)rel * inv_cap) * cap == 0;
        const unsigned mb = __ballot_sync(kFull, brk);
        if (brk) {
            const int k = nrun + __popc(mb & ((1u << lane) - 1u));
            if (k < nrcap) {
                O[k] = val;
                S[k] = i;
            }
        }
        if (RI && valid) RI[i] = nrun + __popc(mb & lane_le) - 1;  // the run this cell belongs to
        if (CP) {
            if (valid) CP[i] = val;
            if (newval) SP[nspan + __popc(nle) - 1] = val;  // span index <= cell index
            nspan += __popc(mnew);
        }
        nrun += __popc(mb);
        n += nvalid;
        if (nvalid < 32) break;
        carried = __shfl_sync(kFull, st, 31);
        prev_bits = __shfl_sync(kFull, bits, 31);
    }
    if (lane == 0 && nrun <= nrcap) S[nrun] = n;
    if (n_out) *n_out = n;
    if (nspan_out) *nspan_out = nspan;
    __syncwarp();
    return nrun;
}

static __device__ int sample_encode_ray(const float *__restrict__ vox, int X, int Y, int Z, const int32_t *pose,
                                        const int32_t *u, int nsamp, int cap, float *O, int *S)
{
    return sample_encode_ray(vox, X, Y, Z, pose, u, nsamp, cap, O, S, nsamp + 1, nullptr, nullptr, nullptr, nullptr);
}

// ---- the fused 3D ray (sampling and evaluation in one warp) --------------------------------------
//
// Per-warp layout: per-cell o / P (CP), f_emp (CF) and C padded by K zeros on both sides (CC), each
// cell_stride floats (absent for Theorem 5's sub-blocks, which always use the runs), then the six
// run arrays sized for the runs the run-pair path can see: a ray takes that path only when
// n >= cell_runlen * n_r, so n_r <= nmax / cell_runlen.

__host__ __device__ inline bool thm5_of(const DevParams &p) { return p.variant == FSMI_APPROX && p.approx_reading == 0; }
__host__ __device__ inline int ray3d_cell_stride(const DevParams &p) { return ((p.nmax + 2 * p.K + 2) + 3) & ~3; }
__host__ __device__ inline int ray3d_nrcap(const DevParams &p)
{
    const int T = p.cell_runlen > 0 ? p.cell_runlen : 1;
    return thm5_of(p) ? p.nmax : min(p.nmax, p.nmax / T + 2);
}
__host__ __device__ inline int ray3d_run_stride(const DevParams &p) { return ((ray3d_nrcap(p) + 2) + 3) & ~3; }
// Per-warp floats of the fused 3D path. The others: [CP | CF | CC | six run arrays]. Theorem 5 (all
// runs stored): [S | O | four cell-stride arrays], the four holding CP, CF, CC and the cells' run
// indices for the cell form, or the run arrays X, A, F, L for the run pairs.
__host__ __device__ inline int ray3d_warp_floats(const DevParams &p)
{
    return thm5_of(p) ? 2 * ray3d_run_stride(p) + 4 * ray3d_cell_stride(p)
                      : 3 * ray3d_cell_stride(p) + 6 * ray3d_run_stride(p);
}

// Which evaluation paths a fused-ray kernel is compiled with: both (the variant read at run time),
// Theorem 5's sub-blocks only, or the others (cell-level convolution and all run pairs) only.
enum { kRay3dAny = 0, kRay3dThm5 = 1, kRay3dOther = 2 };

// The cells' gains f(delta_occ, o) (Gk) and f(delta_emp, o) (Gf) of a sampled ray: the nspan spans
// of equal values (their values in Gf[0 .. nspan), from sampling) get both gains once, stored in
// place at Gk[k] and Gf[k]; then every cell takes its span's pair, the chunks of 32 cells from the
// last down, each reading before any lane writes: cell i's span index is at most i, so a chunk
// only overwrites entries that no cell below it reads. A cell starts a span where its value's bits
// differ from the previous cell's, as in the sampling.
__device__ __forceinline__ void span_gains(const DevParams &p, const float *CP, float *Gk, float *Gf, int n, int nspan)
{
    const int lane = lane_id();
    for (int k = lane; k < nspan; k += 32) {
        float fo, fe;
        rle_gains(p, Gf[k], fo, fe);
        Gk[k] = fo;
        Gf[k] = fe;
    }
    __syncwarp();
    const unsigned lane_le = 0xffffffffu >> (31 - lane);
    int above = nspan;  // spans that start in the chunks above the current one, counted from the end
    for (int base = ((n - 1) >> 5) << 5; base >= 0; base -= 32) {
        const int i = base + lane;
        const bool in = i < n;
        const bool start = in && (i == 0 || __float_as_uint(CP[i]) != __float_as_uint(CP[i - 1]));
        const unsigned m = __ballot_sync(kFull, start);
        above -= __popc(m);  // now: spans that start before this chunk
        const int k = above + __popc(m & lane_le) - 1;
        float go = 0.0f, ge = 0.0f;
        if (in) {
            go = Gk[k];
            ge = Gf[k];
        }
        __syncwarp();
        if (in) {
            Gk[i] = go;
            Gf[i] = ge;
        }
        __syncwarp();
    }
}

// Samples, encodes and evaluates one ray into the warp's region `w` (ray3d_warp_floats floats);
// returns the MI (warp-reduced) and the run count in *nr_out. MODE must agree with thm5_of(p).
template <int MODE>
__device__ __forceinline__ float ray_mi_fused(const float *vox, int X, int Y, int Z, const int32_t *pose,
                                              const int32_t *u, int nsamp, const DevParams &p, const float2 *tab,
                                              const float *gtab, int K, float *w, int *nr_out)
{
    const int lane = lane_id();
    const bool thm5 = MODE == kRay3dAny ? thm5_of(p) : MODE == kRay3dThm5;
    const int cst = ray3d_cell_stride(p), rst = ray3d_run_stride(p);
    float *CP, *CF, *CC;
    int *RI = nullptr;
    RunSmem r;
    if (thm5) {
        float *c4 = w + 2 * rst;
        CP = c4;
        CF = c4 + cst;
        CC = c4 + 2 * cst;
        RI = (int *)(c4 + 3 * cst);
        r.S = (int *)w;
        r.O = w + rst;
        r.X = CP;
        r.A = CF;
        r.F = CC;
        r.L = RI;
    } else {
        CP = w;
        CF = w + cst;
        CC = w + 2 * cst;
        r = run_smem(w + 3 * cst, rst);
    }
    int n = 0, nspan = 0;
    const int nr = sample_encode_ray(vox, X, Y, Z, pose, u, nsamp, p.run_cap, r.O, r.S, ray3d_nrcap(p), &n, CP, CF,
                                     &nspan, RI);
    *nr_out = nr;
    if (nr <= 0) return 0.0f;
    float v;
    if (n < p.cell_runlen * nr) {
        // eq. eqn_from_fsmi on the virtual cells: Algorithms 2 and 3, then the banded convolution
        // (Theorem 5: over each first-hit cell's window of kept pairs)
        if (!thm5) {
            for (int i = lane; i < K; i += 32) {
                CC[i] = 0.0f;
                CC[K + n + i] = 0.0f;
            }
        }
        span_gains(p, CP, CC + K, CF, n, nspan);
        cell_prefixes(CP, CC + K, CF, n, false);  // CP = P(e_j), CC[K + k] = C_k, CC[K + n] = 0
        if (thm5) {  // RI was filled while sampling
            v = MODE == kRay3dThm5 && K == 15 ? window_conv_k<15>(CP, CC, gtab, n, r.S, RI, p.trunc)
                                               : window_conv(CP, CC, gtab, K, n, r.S, RI, p.trunc);
        } else {
            v = band_conv<MODE == kRay3dOther>(CP, CC, gtab, K, n);
        }
    } else {  // here n_r <= nrcap, so every run was stored
        run_starts(r, nr, true);
        run_prefixes(r, nr, p);
        v = thm5 ? pairs_thm5(r, nr, tab, K, p.trunc) : pairs_all(r, nr, tab, K);
    }
    return warp_sum(v);
}

// pose and ray of batch item `ray` = pose * R + r (a 32-bit division when ray fits, the common case)
__device__ __forceinline__ void split_ray(long long ray, int R, int &pi, int &ri)
{
    if (ray <= 0x7fffffffLL) {
        pi = (int)((unsigned)ray / (unsigned)R);
        ri = (int)((unsigned)ray - (unsigned)pi * (unsigned)R);
    } else {
        pi = (int)(ray / R);
        ri = (int)(ray % R);
    }
}

// ray = pose * R + r of a batch
__device__ __forceinline__ int sample_encode(const Vox3D &v, long long ray, int nsamp, int cap, float *O, int *S)
{
    int pi, ri;
    split_ray(ray, v.R, pi, ri);
    return sample_encode_ray(v.vox, v.X, v.Y, v.Z, v.poses + 12 * (size_t)pi, v.dirs + 3 * (size_t)ri, nsamp, cap, O,
                             S);
}

// ---- kernels -----------------------------------------------------------------------------------

struct TabSpec {
    int kind, H, band, K;
    double sigma;
};

__host__ __device__ inline TabSpec table_spec(const DevParams &p)
{
    TabSpec t;
    t.sigma = p.sigma;
    t.H = p.H;
    t.band = -1;
    t.K = p.K;
    if (p.variant == FSMI_UNIFORM) {
        t.kind = 2;
    } else {
        t.kind = p.g_kernel == FSMI_G_ERF ? 1 : 0;
        if (p.variant == FSMI_APPROX && p.approx_reading == 1) t.band = p.trunc;
    }
    return t;
}

// shared memory: [table float2 (2K+2)] [g scratch double (K+1)] [g float (2K+1)] [per-warp arrays]
__host__ __device__ inline size_t rle_table_bytes(int K)
{
    return ((size_t)(2 * K + 2) * sizeof(float2) + (size_t)(2 * K + 1) * sizeof(float) + 15) & ~(size_t)15;
}

// Shared-memory layout of the RLE evaluation kernels: the block's kernel table, then each warp's
// kArraysRLE arrays of `stride` floats.
struct RleBlock {
    TabSpec ts;
    float2 *tab;
    float *gtab;
    float *base;
};

__device__ __forceinline__ RleBlock rle_block(unsigned char *smem_raw, const DevParams &p, const RleTable &t,
                                              int warp_floats)
{
    RleBlock rb;
    rb.ts = table_spec(p);
    rb.tab = (float2 *)smem_raw;
    rb.gtab = (float *)(smem_raw + (size_t)(2 * rb.ts.K + 2) * sizeof(float2));
    load_table(rb.tab, rb.gtab, rb.ts.K, t);
    rb.base = (float *)(smem_raw + rle_table_bytes(rb.ts.K)) + (size_t)(threadIdx.x >> 5) * warp_floats;
    return rb;
}

// sampling, encoding and evaluation of one 3D ray (= pose * R + r), fused layout; WIDE: the batch
// has more than 2^31 - 1 rays (64-bit index division), else a 32-bit one
template <int MODE, bool WIDE>
__device__ __forceinline__ void eval_ray_3d(const Vox3D &vx, const DevParams &p, const RleBlock &rb,
                                            long long ray, float *__restrict__ out, int32_t *__restrict__ nruns)
{
    int pi, ri;
    if (WIDE) {
        pi = (int)(ray / vx.R);
        ri = (int)(ray % vx.R);
    } else {
        pi = (int)((unsigned)ray / (unsigned)vx.R);
        ri = (int)((unsigned)ray - (unsigned)pi * (unsigned)vx.R);
    }
    int nr = 0;
    const float I = ray_mi_fused<MODE>(vx.vox, vx.X, vx.Y, vx.Z, vx.poses + 12 * (size_t)pi, vx.dirs + 3 * (size_t)ri, p.nmax,
                                 p, rb.tab, rb.gtab, rb.ts.K, rb.base, &nr);
    if (lane_id() == 0) {
        out[ray] = I;
        if (nruns) nruns[ray] = nr;
    }
    __syncwarp();
}

// evaluation of one run-length-encoded ray given in CSR form
__device__ __forceinline__ void eval_ray_rle(const int32_t *__restrict__ off, const float *__restrict__ ro,
                                             const uint8_t *__restrict__ rl, const DevParams &p, const RleBlock &rb,
                                             int stride, long long ray, float *__restrict__ out, int *status)
{
    const int lane = lane_id();
    const RunSmem r = run_smem(rb.base, stride);
    const int b = off[ray];
    const int nr = off[ray + 1] - b;
    bool bad = b < 0 || nr < 0 || nr > p.nmax;
    int cells = 0;
    if (!bad) {
        for (int u = lane; u < nr; u += 32) {
            const int L = rl[b + u];
            r.O[u] = __ldg(ro + b + u);
            r.L[u] = L;
            cells += L;
            bad |= (L == 0);
        }
        cells = __reduce_add_sync(kFull, cells);
        bad = __any_sync(kFull, bad) || cells > p.nmax;
    }
    __syncwarp();
    if (bad) {
        if (lane == 0) {
            out[ray] = __int_as_float(0x7fc00000);
            set_status(status, FSMI_STATUS_BAD_BEAM);
        }
        __syncwarp();
        return;
    }
    const float I = ray_mi(rb.base, stride, nr, p, rb.tab, rb.gtab, rb.ts.K, false);
    if (lane == 0) out[ray] = I;
    __syncwarp();
}

}  // namespace fsmi
