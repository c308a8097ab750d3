// 2D hot path (device code shared by the 2D and mixed kernels): fixed-point ray traversal,
// first-hit probabilities, C_k and the FSMI / Approx-FSMI / Uniform-FSMI pair sums, one warp per beam.
//
// Per beam (Section 3): the traversal lists the cells the beam crosses with entry distances
// l_1 = 0 < l_2 < ... and end l_{n+1}; Algorithm 2 gives P(e_j) = o_j prod_{i<j}(1 - o_i);
// Algorithm 3 gives C_k = sum_{i<k} f(delta_emp, r_i) + f(delta_occ, r_k); the variant then sums
//   FSMI (Theorem 1):         sum_j P(e_j) sum_{k=1..n} C_k G_{k,j}
//   Approx (eq. fsmi_approx): the same with |k - j| <= Delta
//   Uniform (Algorithm 4):    sum_j P(e_j) (D_{min(n,j+H)} - D_{max(0,j-H-1)}) / (2H + 1)
//
// The Gaussian pair sum is evaluated per first-hit cell j in boundary form (summation by parts):
//   S_j = sum_k C_k (Phi(x_{k+1}) - Phi(x_k)) = C_j + sum_{m=1}^{n+1} (C_m - C_{m-1}) sgn(x_m) T(|x_m|)
// with x_m = (l_m - mu_j) / sigma, C_0 = C_{n+1} = 0 and T the upper Gaussian tail. Every term is
// a tail mass, so no difference of two values near 1 is formed in FP32, and each (j, m) pair costs
// one tail evaluation (gauss_tail.cuh) instead of the two Phi values of G_{k,j}. The sign is taken
// from the indices (boundaries m <= j lie before the centre of cell j), not from the FP32
// difference, which is 0 for a cell shorter than the FP32 resolution of its distance.
#pragma once

#include "../../include/fsmi.h"
#include "fsmi_device.cuh"
#include "dda2d.cuh"
#include "fsmi_internal.h"
#include "gauss_tail.cuh"

namespace fsmi {

// ---- pair sums ------------------------------------------------------------------------------------

// per-warp shared arrays, in units of `stride` floats: l, C, P, scratch (ids / f_emp / D / dC)
constexpr int kArrays2D = 4;
// Padding boundaries before index 0 and after index n + 1 of l and dC (l = -+3e30, dC = 0: their
// terms are exactly zero), so that the exact window loops can run past a beam's ends.
constexpr int kPad2D = 32;

// Floats between consecutive arrays for beams of up to nmax cells (n + 2 boundaries + padding).
__host__ __device__ constexpr int stride_2d(int nmax) { return ((nmax + 2 + kPad2D) + 3) & ~3; }
// Floats of one warp's arrays: kArrays2D strides and the front padding of l and dC.
__host__ __device__ constexpr int warp_floats_2d(int stride) { return kArrays2D * stride + 2 * kPad2D; }

// One warp's arrays in its region `base` (16-byte aligned): [pad | l | C | P | pad | scratch].
__device__ __forceinline__ void carve_2d(float *base, int stride, float *&sl, float *&sc, float *&sp, float *&sx)
{
    sl = base + kPad2D;
    sc = sl + stride;
    sp = sc + stride;
    sx = sp + stride + kPad2D;
}
// internal variant id of the full n(n+1) exact sweep (FSMI_FLAG_FULL_SWEEP)
constexpr int kExactFullSweep = 3;

enum { kSrcMap = 0, kSrcBeams = 1, kSrcSets = 2, kSrcTraj = 3 };

struct Src2D {
    // map source (kSrcMap, kSrcSets)
    const float *map;
    int W, H;
    const int32_t *poses;
    int P;
    const int32_t *dirs;
    int B;
    const float4 *gains;  // optional per-map-cell (o, f_occ, f_emp, 0)
    // explicit-beam source (kSrcBeams)
    const int32_t *off;
    const float *o;
    const float *l;
    const float *lend;
    // candidate sets (kSrcSets): device array of nsets descriptors
    const fsmi_set_2d *sets;
    int nsets;
    // trajectories (kSrcTraj, poses and beams as kSrcMap): states traj_off[t] .. traj_off[t+1]-1,
    // stamp[t][cell] = first state of trajectory t whose beams visit the cell
    const int32_t *traj_off;
    int T;
    const int32_t *stamp;
};

// One register-blocked pass of the exact pair sum over scaled distances: each lane owns J
// first-hit slots j = jb + lane + 32 t and streams every boundary m = 0..n from shared memory.
// Slot n is the no-return event when e0 is set (centre mu0, C_0 = 0). Terms of even and odd m
// accumulate separately, each in increasing m, and are added at the end (the order the window
// sum uses, so that the two agree bit for bit).
template <int J>
__device__ __forceinline__ float exact_pass(const float *sl, const float *sc, const float *sp, int n, int jb,
                                            bool e0, float pe0, float mu0)
{
    const int lane = lane_id();
    float mu[J], acc[J], acc1[J];
    int mid[J];  // boundaries m < mid lie before the centre
#pragma unroll
    for (int t = 0; t < J; ++t) {
        const int j = jb + lane + 32 * t;
        mu[t] = (j < n) ? 0.5f * (sl[j] + sl[j + 1]) : ((j == n && e0) ? mu0 : 3.0e30f);
        mid[t] = (j < n) ? j + 1 : 0;
        acc[t] = 0.0f;
        acc1[t] = 0.0f;
    }
    float cprev = 0.0f;
    for (int m = 0; m <= n; ++m) {
        const float lm = sl[m];
        const float cm = sc[m];  // sc[n] = 0 (C_{n+1})
        const float dc = cm - cprev;
        cprev = cm;
        if (m & 1) {
#pragma unroll
            for (int t = 0; t < J; ++t) acc1[t] = fmaf(m < mid[t] ? -dc : dc, gauss_tail(lm - mu[t]), acc1[t]);
        } else {
#pragma unroll
            for (int t = 0; t < J; ++t) acc[t] = fmaf(m < mid[t] ? -dc : dc, gauss_tail(lm - mu[t]), acc[t]);
        }
    }
    float r = 0.0f;
#pragma unroll
    for (int t = 0; t < J; ++t) {
        const int j = jb + lane + 32 * t;
        const float a = acc[t] + acc1[t];
        if (j < n)
            r = fmaf(sp[j], sc[j] + a, r);
        else if (j == n && e0)
            r = fmaf(pe0, a, r);
    }
    return r;
}

__device__ __forceinline__ float exact_sum(const float *sl, const float *sc, const float *sp, int n, bool e0,
                                           float pe0, float mu0)
{
    const int nslots = n + (e0 ? 1 : 0);
    float r = 0.0f;
    for (int jb = 0; jb < nslots; jb += 32 * 16) {
        const int cnt = min(16, (nslots - jb + 31) >> 5);
        switch (cnt) {
#define FSMI_CASE(J) \
    case J: r += exact_pass<J>(sl, sc, sp, n, jb, e0, pe0, mu0); break;
            FSMI_CASE(1) FSMI_CASE(2) FSMI_CASE(3) FSMI_CASE(4) FSMI_CASE(5) FSMI_CASE(6) FSMI_CASE(7) FSMI_CASE(8)
            FSMI_CASE(9) FSMI_CASE(10) FSMI_CASE(11) FSMI_CASE(12) FSMI_CASE(13) FSMI_CASE(14) FSMI_CASE(15)
            FSMI_CASE(16)
#undef FSMI_CASE
            default: break;
        }
    }
    return r;
}

// Largest scaled distance whose tail is not flushed to zero: beyond |d| = 11.3 the factor
// 2^(-d^2) <= 2^(-127.69) is subnormal and ex2.approx.ftz returns exactly 0, so the term is +-0.
constexpr float kTailCut = 11.3f;
// Default window of the exact sum: T(4.81) = 7.4e-9 < 2^-27. Boundaries come at most two per
// major-axis crossing interval (scaled length >= cs = sqrt(log2 e) / (sigma sqrt 2)), so the terms
// skipped on one side weigh at most 2 T(4.81) / (1 - 2^(-9.62 cs)) times max |C_m - C_{m-1}|:
// at most 2^-24 of it (one FP32 ulp) for sigma up to 19 cells (1.01 x 2^-24 at 20), below 2^-25
// for sigma <= 2.
constexpr float kTailCutDefault = 4.81f;

// Boundary terms of one first-hit cell with centre mu over the pairs (m, m + 1), m = m0, m0 + 2,
// ... < end (m0, nb and end even, m0 <= nb <= end), so that every term goes through the packed
// tail; the pairs below nb lie before the centre, the pair at nb straddles it when mid is odd.
// A boundary m < mid lies before the centre: -dC_m T(mu - l_m); above it +dC_m T(l_m - mu).
// Padding boundaries (l = -+3e30, dC = 0) give exact zeros. Returns the packed sums over even and
// odd m, each added in increasing m.
#ifndef FSMI_PAIR_UNROLL
#define FSMI_PAIR_UNROLL 4
#endif
constexpr int kPairUnroll = FSMI_PAIR_UNROLL;  // boundary pairs in flight per lane, exact window loop

__device__ __forceinline__ f32x2 window_terms(const float *sl, const float *sdc, int m, int nb, int end, int mid, float mu)
{
    const f32x2 mu2 = pack2(mu, mu);
    f32x2 acc = pack2(0.0f, 0.0f);
#pragma unroll kPairUnroll
    for (; m < nb; m += 2) {  // pairs (m, m + 1) with m + 1 < mid
        const f32x2 L = *reinterpret_cast<const f32x2 *>(sl + m);
        const f32x2 dc = *reinterpret_cast<const f32x2 *>(sdc + m);
        acc = fma2(dc, gauss_tail2p<true>(sub2(mu2, L)), acc);
    }
    if (m < end) {  // first pair at or above the centre; m lies below it when m == mid - 1
        const float2 L = *reinterpret_cast<const float2 *>(sl + m);
        const float2 dc = *reinterpret_cast<const float2 *>(sdc + m);
        const bool below = m == mid - 1;
        const float d0 = below ? mu - L.x : L.x - mu;
        const float c0 = below ? -dc.x : dc.x;
        acc = fma2(pack2(c0, dc.y), gauss_tail2p<false>(pack2(d0, L.y - mu)), acc);
        m += 2;
    }
#pragma unroll kPairUnroll
    for (; m < end; m += 2) {
        const f32x2 L = *reinterpret_cast<const f32x2 *>(sl + m);
        const f32x2 dc = *reinterpret_cast<const f32x2 *>(sdc + m);
        acc = fma2(dc, gauss_tail2p<false>(sub2(L, mu2)), acc);
    }
    return acc;
}

// Exact pair sum over the boundaries within the window: for slot j at least the m with
// |l_m - mu_j| < cut (scaled) are visited, in increasing m. With cut = kTailCut every non-zero
// term of the full sweep is added in the same order and the FP32 result is the same bit for bit;
// with kTailCutDefault the terms skipped are below 2^-27 of their weights.
// The 32 slots of a round run the same number of pairs below and above their centres: the
// fewest pairs G that cover every slot's window on that side. A slot whose window is shorter adds
// the next boundaries beyond it, which are terms of the full sum too (or padding with weight 0),
// so that no lane leaves the unrolled loops at a different point than the others. No window end is
// searched for: with the pairs below the centre starting at nb - 2G, a slot is covered when the
// boundary before that start lies below mu - cut (one shared load per lane and trial G), and the
// trials start from the previous round's G, which changes little along a beam.
// sdc[m] = C_m - C_{m-1} for m = 0..n; sl and sdc padded by kPad2D entries on both sides.
__device__ __forceinline__ float exact_window_sum(const float *sl, const float *sdc, const float *sc,
                                                  const float *sp, int n, bool e0, float pe0, float mu0, float cut)
{
    const int nslots = n + (e0 ? 1 : 0);
    // first trial: about cut x (boundaries per unit of scaled distance) boundaries on each side
    const float span = sl[n] - sl[0];
    const float per = span > 0.0f ? (float)n / span : 0.0f;
    int GN = (int)fminf(cut * per, (float)(n + 1)) >> 1, GP = GN;
    const int mtop = (n + 1 + kPad2D) & ~1;  // pairs (m, m + 1) stay below n + 2 + kPad2D
    float r = 0.0f;
    for (int jb = 0; jb < nslots; jb += 32) {
        const int j = jb + lane_id();
        const bool act = j < nslots;
        float mu = 0.0f, Cj = 0.0f, Pj = 0.0f;
        int mid = 0;
        if (act && j < n) {
            mu = 0.5f * (sl[j] + sl[j + 1]);
            Cj = sc[j];
            Pj = sp[j];
            mid = j + 1;
        } else if (act) {  // the no-return slot: centre before l_0, every boundary above it
            mu = mu0;
            Pj = pe0;
        }
        const int nb = mid & ~1;  // pairs (m, m + 1) with m + 1 < mid end here
        const float below = mu - cut, above = mu + cut;
        // below the centre: covered at G when every boundary before nb - 2G lies below mu - cut
        // (true for every G once nb - 2G <= 0, so both loops end)
        auto neg_ok = [&](int G) {
            const int m = nb - 2 * G;
            return !act || m <= 0 || sl[m - 1] < below;
        };
        // above it: covered when every boundary from nb + 2 + 2G on lies at or beyond mu + cut
        // (true once that index passes n)
        auto pos_ok = [&](int G) {
            const int e = nb + 2 + 2 * G;
            return !act || e > n || sl[e] >= above;
        };
        if (__all_sync(kFull, neg_ok(GN))) {
            while (GN > 0 && __all_sync(kFull, neg_ok(GN - 1))) --GN;
        } else {
            do ++GN;
            while (!__all_sync(kFull, neg_ok(GN)));
        }
        if (__all_sync(kFull, pos_ok(GP))) {
            while (GP > 0 && __all_sync(kFull, pos_ok(GP - 1))) --GP;
        } else {
            do ++GP;
            while (!__all_sync(kFull, pos_ok(GP)));
        }
        const int m0 = act ? max(nb - 2 * GN, -kPad2D) : 0;
        const int end = act ? min(nb + 2 + 2 * GP, mtop) : 0;
        float a0, a1;
        unpack2(window_terms(sl, sdc, m0, nb, end, mid, mu), a0, a1);
        r = fmaf(Pj, Cj + (a0 + a1), r);
    }
    return r;
}

// Boundary terms m in [a, b) on one side of a first-hit cell's centre, added to acc: before the
// centre (NEG) -dC_m T(mu - l_m), after it +dC_m T(l_m - mu). Pairs at even m go through the
// packed tail; an odd first or last boundary is evaluated alone.
template <bool NEG>
__device__ __forceinline__ float side_terms(const float *sl, const float *sdc, int a, int b, float mu, float acc)
{
    int m = a;
    if (m < b && (m & 1)) {
        acc = fmaf(NEG ? -sdc[m] : sdc[m], gauss_tail(NEG ? mu - sl[m] : sl[m] - mu), acc);
        ++m;
    }
    const f32x2 mu2 = pack2(mu, mu);
    f32x2 acc2 = pack2(0.0f, 0.0f);
#pragma unroll 2
    for (; m + 1 < b; m += 2) {
        const f32x2 L = *reinterpret_cast<const f32x2 *>(sl + m);
        const f32x2 dc = *reinterpret_cast<const f32x2 *>(sdc + m);
        acc2 = fma2(dc, gauss_tail2p<NEG>(NEG ? sub2(mu2, L) : sub2(L, mu2)), acc2);
    }
    float a0, a1;
    unpack2(acc2, a0, a1);
    acc += a0 + a1;
    if (m < b) acc = fmaf(NEG ? -sdc[m] : sdc[m], gauss_tail(NEG ? mu - sl[m] : sl[m] - mu), acc);
    return acc;
}

// Approx-FSMI: for slot j the band k in [klo, khi] = [j - Delta, j + Delta] n [0, n-1] (0-based),
// i.e. boundaries m in [klo, khi + 1] with C' = C on the band and 0 outside it: the band edges
// weigh C_klo and -C_khi, the interior C_m - C_{m-1} (sdc).
__device__ __forceinline__ float approx_sum(const float *sl, const float *sc, const float *sdc, const float *sp,
                                            int n, bool e0, float pe0, float mu0, int D)
{
    const int nslots = n + (e0 ? 1 : 0);
    float r = 0.0f;
    for (int j = lane_id(); j < nslots; j += 32) {
        float mu, Cj, Pj;
        int klo, khi;
        if (j < n) {
            mu = 0.5f * (sl[j] + sl[j + 1]);
            Cj = sc[j];
            Pj = sp[j];
            klo = max(0, j - D);
            khi = min(n - 1, j + D);
        } else {  // e_0 at virtual index 0: paper band k in [1, Delta]
            mu = mu0;
            Cj = 0.0f;
            Pj = pe0;
            klo = 0;
            khi = min(n - 1, D - 1);
        }
        const int mid = (j < n) ? j + 1 : 0;  // boundaries m < mid lie before the centre
        float acc = 0.0f;
        if (klo <= khi) {  // an empty band (e_0 with Delta = 0) adds nothing
            const float clo = sc[klo], chi = sc[khi];
            acc = fmaf(klo < mid ? -clo : clo, gauss_tail(sl[klo] - mu), acc);
            const int split = min(max(mid, klo + 1), khi + 1);
            acc = side_terms<true>(sl, sdc, klo + 1, split, mu, acc);
            acc = side_terms<false>(sl, sdc, split, khi + 1, mu, acc);
            acc = fmaf(khi + 1 < mid ? chi : -chi, gauss_tail(sl[khi + 1] - mu), acc);
        }
        r = fmaf(Pj, Cj + acc, r);
    }
    return r;
}

// Uniform-FSMI (Algorithm 4) from D = inclusive prefix of C (sd), with Algorithm 4's clamps.
__device__ __forceinline__ float uniform_sum(const float *sd, const float *sp, int n, bool e0, float pe0, int H,
                                             float inv_2h1)
{
    float r = 0.0f;
    for (int j = lane_id(); j < n; j += 32) {
        const int hi = min(n - 1, j + H);
        const int lo = j - H - 1;
        const float S = (sd[hi] - (lo >= 0 ? sd[lo] : 0.0f)) * inv_2h1;
        r = fmaf(sp[j], S, r);
    }
    if (e0 && lane_id() == 0) {
        const int hi = min(n - 1, H - 1);
        if (hi >= 0) r = fmaf(pe0, sd[hi] * inv_2h1, r);
    }
    return r;
}

#ifndef FSMI_MIN_BLOCKS_2D
#define FSMI_MIN_BLOCKS_2D 4  // resident 8-warp blocks per SM requested from the register allocator (64 registers)
#endif

// the candidate set holding flat beam index `beam` (sets sorted by beam_offset)
__device__ __forceinline__ int set_of(const fsmi_set_2d *sets, int nsets, long long beam)
{
    int lo = 0, len = nsets;
    while (len > 0) {
        const int half = len >> 1;
        if (__ldg(&sets[lo + half].beam_offset) <= beam) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo - 1;
}

// the trajectory holding pose p: t with traj_off[t] <= p < traj_off[t+1], or -1
__device__ __forceinline__ int traj_of(const int32_t *traj_off, int T, int p)
{
    int lo = 0, len = T + 1;  // last index with traj_off[idx] <= p
    while (len > 0) {
        const int half = len >> 1;
        if (__ldg(traj_off + lo + half) <= p) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    const int t = lo - 1;
    return (t >= 0 && t < T && p < __ldg(traj_off + t + 1)) ? t : -1;
}

// Cells of one beam on the map: traversal from `pose` along the sensor-frame direction (ux, uy)
// up to rfix (Q16) / rend, then per cell o (sp), f(delta_occ, o) (sc), f(delta_emp, o) (sx) and
// the entry distances (sl). With TRAJ, cells whose visit stamp is below `state` keep o but lose
// their gains (Section 2.4). Returns n, or -1 if the beam has more than cap cells.
template <bool TRAJ>
__device__ __forceinline__ int beam_cells(const float *__restrict__ map, int W, int H, const float4 *__restrict__ gains,
                                          const int32_t *pose, int ux, int uy, long long rfix, float rend, int cap,
                                          const DevParams &p, int state, const int32_t *stamps, float *sl, float *sc,
                                          float *sp, float *sx, int *status)
{
    const int lane = lane_id();
    int dx, dy;
    beam_dir(pose, ux, uy, dx, dy);
    const int n = dda_warp(W, H, pose[0], pose[1], dx, dy, rfix, rend, cap, (int *)sx, sl);
    if (n < 0) return -1;
    const unsigned ncell = (unsigned)W * (unsigned)H;
    bool bad = false;
    if (gains) {
        for (int i = lane; i < n; i += 32) {
            const unsigned id = (unsigned)((const int *)sx)[i];
            bad |= id >= ncell;  // cannot happen for a consistent traversal; never read out of bounds
            float4 v = id < ncell ? __ldg(gains + id) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (TRAJ && id < ncell && __ldg(stamps + id) < state) v.y = v.z = 0.0f;
            sp[i] = v.x;
            sc[i] = v.y;
            sx[i] = v.z;
        }
    } else {
        for (int i = lane; i < n; i += 32) {
            const unsigned id = (unsigned)((const int *)sx)[i];
            bad |= id >= ncell;
            const float o = id < ncell ? __ldg(map + id) : 0.0f;
            // a cell already counted by an earlier state of the trajectory (Section 2.4) still
            // stops the beam with probability o but adds no information
            const bool counted = TRAJ && id < ncell && __ldg(stamps + id) < state;
            sp[i] = o;
            sc[i] = counted ? 0.0f : cell_gain(p.docc, o);
            sx[i] = counted ? 0.0f : cell_gain(p.demp, o);
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) set_status(status, FSMI_STATUS_INTERNAL);
    __syncwarp();
    return n;
}

// The variant's mutual information of one beam of n cells held in shared memory (sl: n + 1
// distances, sp: o, sc: f_occ, sx: f_emp): Algorithm 2, Algorithm 3 (4), then the pair sum.
template <int VAR>
__device__ __forceinline__ float beam_sum(const DevParams &p, int n, float *sl, float *sc, float *sp, float *sx)
{
    const int lane = lane_id();
    const bool e0 = p.e0 != 0;
    const float cs = p.inv_s2 * (float)kSqrtLog2e;  // distance -> tail variable
    float I = 0.0f;
    if (n > 0) {
        if (VAR != FSMI_UNIFORM) {
            for (int i = lane; i <= n; i += 32) sl[i] *= cs;
        }
        const float pe0 = cell_prefixes(sp, sc, sx, n, VAR == FSMI_UNIFORM);
        const float mu0 = sl[0] - 0.5f * cs;  // e_0 centre, l_1 - 1/2 (scaled)
        if (VAR == kExactFullSweep) I = exact_sum(sl, sc, sp, n, e0, pe0, mu0);
        if (VAR == FSMI_EXACT) {
            for (int m = lane; m <= n; m += 32) sx[m] = sc[m] - (m > 0 ? sc[m - 1] : 0.0f);
            for (int i = lane; i < kPad2D; i += 32) {  // padding boundaries on both sides, weight 0
                sl[-1 - i] = -3.0e30f;
                sx[-1 - i] = 0.0f;
                sl[n + 1 + i] = 3.0e30f;
                sx[n + 1 + i] = 0.0f;
            }
            __syncwarp();
            I = exact_window_sum(sl, sx, sc, sp, n, e0, pe0, mu0,
                                 (p.flags & FSMI_FLAG_FULL_WINDOW) ? kTailCut : kTailCutDefault);
        }
        if (VAR == FSMI_APPROX) {
            for (int m = lane; m <= n; m += 32) sx[m] = sc[m] - (m > 0 ? sc[m - 1] : 0.0f);
            __syncwarp();
            I = approx_sum(sl, sc, sx, sp, n, e0, pe0, mu0, p.trunc);
        }
        if (VAR == FSMI_UNIFORM) I = uniform_sum(sx, sp, n, e0, pe0, p.H, p.inv_2h1);
        I = warp_sum(I);
    }
    return I;
}

__device__ __forceinline__ void store_nan(float *out, long long i, int *status, int bits)
{
    if (lane_id() == 0) {
        out[i] = __int_as_float(0x7fc00000);
        set_status(status, bits);
    }
    __syncwarp();
}

// One beam: traversal (or explicit cells), gains, prefixes, the variant's pair sum, store.
template <int VAR, int SRC>
__device__ __forceinline__ void eval_beam(const Src2D &src, const DevParams &p, long long beam, float *sl, float *sc,
                                          float *sp, float *sx, float *__restrict__ out, int *status)
{
    const int lane = lane_id();
    int n;
    if (SRC != kSrcBeams) {
        const int32_t *pose;
        int ux, uy;
        int state = 0;                   // kSrcTraj: state index within the trajectory
        const int32_t *stamps = nullptr;  // kSrcTraj: the trajectory's visit stamps
        long long rfix = p.rfix;
        float rend = p.rend;
        if (SRC == kSrcMap || SRC == kSrcTraj) {
            const int pi = (int)(beam / src.B), bi = (int)(beam % src.B);
            pose = src.poses + 4 * (size_t)pi;
            ux = src.dirs[2 * bi];
            uy = src.dirs[2 * bi + 1];
            if (SRC == kSrcTraj) {
                const int t = traj_of(src.traj_off, src.T, pi);
                if (t < 0) return store_nan(out, beam, status, FSMI_STATUS_BAD_BEAM);  // pose outside every trajectory
                state = pi - __ldg(src.traj_off + t);
                stamps = src.stamp + (size_t)t * src.W * src.H;
            }
        } else {
            const int si = set_of(src.sets, src.nsets, beam);
            bool ok = si >= 0;
            fsmi_set_2d st{};
            if (ok) st = src.sets[si];
            const long long k = beam - st.beam_offset;
            const long long nb = (long long)st.npose * st.nbeam;
            ok = ok && st.npose >= 0 && st.nbeam > 0 && k >= 0 && k < nb;
            long long pi = 0, bi = 0;
            if (ok) {
                pi = st.pose_offset + k / st.nbeam;
                bi = st.dir_offset + k % st.nbeam;
                ok = st.pose_offset >= 0 && st.dir_offset >= 0 && pi < src.P && bi < src.B;
            }
            if (ok) {
                ok = st.max_range > 0.0f && st.max_range <= p.rmax;
                rfix = __double2ll_rn((double)st.max_range * 65536.0);
                rend = (float)((double)rfix * (1.0 / 65536.0));
            }
            if (!ok) return store_nan(out, beam, status, FSMI_STATUS_BAD_BEAM);  // never index with it
            pose = src.poses + 4 * (size_t)pi;
            ux = src.dirs[2 * bi];
            uy = src.dirs[2 * bi + 1];
        }
        n = beam_cells<SRC == kSrcTraj>(src.map, src.W, src.H, src.gains, pose, ux, uy, rfix, rend, p.nmax, p, state,
                                        stamps, sl, sc, sp, sx, status);
        if (n < 0) return store_nan(out, beam, status, FSMI_STATUS_BEAM_OVERFLOW);
    } else {
        const int base = src.off[beam];
        n = src.off[beam + 1] - base;
        if (n < 0 || n > p.nmax) return store_nan(out, beam, status, FSMI_STATUS_BAD_BEAM);
        for (int i = lane; i < n; i += 32) {
            const float o = __ldg(src.o + base + i);
            sl[i] = __ldg(src.l + base + i);
            sp[i] = o;
            sc[i] = cell_gain(p.docc, o);
            sx[i] = cell_gain(p.demp, o);
        }
        if (lane == 0) sl[n] = __ldg(src.lend + beam);
        __syncwarp();
    }
    const float I = beam_sum<VAR>(p, n, sl, sc, sp, sx);
    if (lane == 0) out[beam] = I;
    __syncwarp();
}

}  // namespace fsmi
