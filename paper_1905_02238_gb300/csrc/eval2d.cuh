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

// per-warp shared arrays, in units of `stride` floats: l, scratch (ids / f_emp / D / dC), C, P
constexpr int kArrays2D = 4;
// Padding boundaries before index 0 and after index n + 1 of the exact sum's boundary pairs
// (l = -+3e30, dC = 0: their terms are exactly zero), so that its loops can run past a beam's ends.
constexpr int kPad2D = 32;
constexpr int kPadPairs = kPad2D / 2;

// Floats between consecutive arrays for beams of up to nmax cells (n + 2 boundaries + padding).
__host__ __device__ constexpr int stride_2d(int nmax) { return ((nmax + 2 + kPad2D) + 3) & ~3; }
// Floats of one warp's arrays: kArrays2D strides and the front padding of the boundary pairs.
__host__ __device__ constexpr int warp_floats_2d(int stride) { return kArrays2D * stride + 2 * kPad2D; }

// One warp's arrays in its region `base` (16-byte aligned): [pad | l | scratch | C | P]. The pad,
// l and scratch arrays are contiguous: the exact sum rebuilds them in place as boundary pairs.
__device__ __forceinline__ void carve_2d(float *base, int stride, float *&sl, float *&sc, float *&sp, float *&sx)
{
    sl = base + 2 * kPad2D;
    sx = sl + stride;
    sc = sx + stride;
    sp = sc + stride;
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

// Largest scaled distance whose tail is not flushed to zero: beyond |d| = 11.3 the factor
// 2^(-d^2) <= 2^(-127.69) is subnormal and ex2.approx.ftz returns exactly 0, so the term is +-0.
constexpr float kTailCut = 11.3f;
// Default window of the exact sum: T(4.81) = 7.4e-9 < 2^-27. Boundaries come at most two per
// major-axis crossing interval (scaled length >= cs = sqrt(log2 e) / (sigma sqrt 2)), so the terms
// skipped on one side weigh at most 2 T(4.81) / (1 - 2^(-9.62 cs)) times max |C_m - C_{m-1}|:
// at most 2^-24 of it (one FP32 ulp) for sigma up to 19 cells (1.01 x 2^-24 at 20), below 2^-25
// for sigma <= 2.
constexpr float kTailCutDefault = 4.81f;

// ---- the exact pair sum over boundary pairs ------------------------------------------------------
//
// Boundary pairs: Q[P] = (l_{2P}, l_{2P+1}, dC_{2P}, dC_{2P+1}) with scaled distances l and
// dC_m = C_m - C_{m-1} (C_{-1} = C_n = 0), for P in [-kPadPairs, n / 2 + 1 + kPadPairs); pairs
// past either end of the beam are padding (l = -+3e30, dC = 0). One 16-byte shared load gives a
// pair's two distances and two weights.
//
// Built in place over the traversal's distances sl and the scratch array after them (ids, then
// f_emp, both dead by now), from the top pair down: writing Q[P] overwrites l_{4P} .. l_{4P+3},
// which only Q[2P] and Q[2P+1] read, and those lie higher (P >= 1) or in the same step of 32 pairs,
// whose reads all come before its writes.
__device__ __forceinline__ void build_pairs(float *sl, const float *sc, int n, float cs)
{
    const int lane = lane_id();
    float4 *Q = reinterpret_cast<float4 *>(sl);
    const int pend = (n >> 1) + 1 + kPadPairs;  // pairs 0 .. pend - 1 (the last kPadPairs all padding)
    for (int top = pend; top > 0; top -= 32) {
        const int P = top - 32 + lane;
        float4 v = make_float4(3.0e30f, 3.0e30f, 0.0f, 0.0f);
        if (P >= 0) {
            const int m = 2 * P;
            if (m <= n) {  // l_m, l_{m+1} and C_m, C_{m+1} as 8-byte loads (m even); sc[n] = C_n = 0
                const float2 l2 = *reinterpret_cast<const float2 *>(sl + m);
                const float2 c2 = *reinterpret_cast<const float2 *>(sc + m);
                const float cm = m > 0 ? sc[m - 1] : 0.0f;
                v.x = l2.x * cs;
                v.z = c2.x - cm;
                if (m + 1 <= n) {
                    v.y = l2.y * cs;
                    v.w = c2.y - c2.x;
                }
            }
        }
        __syncwarp();
        if (P >= 0) Q[P] = v;
        __syncwarp();
    }
    if (lane < kPadPairs) Q[-1 - lane] = make_float4(-3.0e30f, -3.0e30f, 0.0f, 0.0f);
    __syncwarp();
}

// Boundary terms of the pairs (m, m + 1), m even, for the first-hit centre mu: below it (NEG)
// -dC_m T(mu - l_m), above it +dC_m T(l_m - mu), two terms per packed operation.
#ifndef FSMI_PAIR_UNROLL
#define FSMI_PAIR_UNROLL 4
#endif
#ifndef FSMI_PAIR2_UNROLL
#define FSMI_PAIR2_UNROLL 2
#endif
constexpr int kPairUnroll = FSMI_PAIR_UNROLL;    // boundary pairs in flight per lane, one slot per lane
constexpr int kPair2Unroll = FSMI_PAIR2_UNROLL;  // the same, two slots per lane (twice the work per pair)

template <bool NEG>
__device__ __forceinline__ f32x2 pair_term(const float4 &q, f32x2 mu2, f32x2 acc)
{
    const f32x2 L = pack2(q.x, q.y), dc = pack2(q.z, q.w);
    return fma2(dc, gauss_tail2p<NEG>(NEG ? sub2(mu2, L) : sub2(L, mu2)), acc);
}

// the pair (m, m + 1) that straddles the centre: m below it, m + 1 above
__device__ __forceinline__ f32x2 straddle_term(const float4 &q, float mu, f32x2 acc)
{
    return fma2(pack2(-q.z, q.w), gauss_tail2p<false>(pack2(mu - q.x, q.y - mu)), acc);
}

// Exact pair sum (Theorem 1) of one beam over the boundary pairs Q: for every first-hit slot j at
// least the boundaries with |l_m - mu_j| < cut (scaled) are visited, in increasing m, even and odd
// m in the two halves of a packed accumulator. With cut = kTailCut every non-zero term of the full
// sweep is added, in the same order, so the FP32 result equals the full sweep (cut = +inf) bit for
// bit; with kTailCutDefault the terms skipped are below 2^-27 of their weights.
//
// Slots go in rounds of 64 while more than 32 remain: lane i takes the adjacent slots A = jb + 2i
// and B = A + 1 and evaluates both against each pair it loads. Pairs below A (m < A) lie below both
// centres, the pair at m = A straddles A's centre and lies below B's, pairs from A + 2 on lie above
// both. The last <= 32 slots (and the no-return slot n when e0 is set: centre mu0 before l_0, every
// boundary above it) go one per lane. In every round all lanes run the same number of pairs below
// and above (the fewest that cover every window of the round), so that no lane leaves the unrolled
// loops early; a lane whose window is shorter adds boundaries beyond it, which are terms of the
// full sum as well (or padding). The counts come from coverage trials that start from the previous
// round's: below, a count G covers a slot when the boundary just before the loop's first pair lies
// below mu - cut; above, when the boundary just after its last pair lies at or beyond mu + cut.
__device__ __forceinline__ float exact_pairs_sum(const float4 *Q, const float *sc, const float *sp, int n, bool e0,
                                                 float pe0, float mu0, float cut)
{
    const int lane = lane_id();
    const float *Qf = reinterpret_cast<const float *>(Q);
    auto lq = [&](int m) { return Qf[4 * (m >> 1) + (m & 1)]; };  // l_m (m >> 1 floors negative m)
    const int nslots = n + (e0 ? 1 : 0);
    const int mtop = ((n >> 1) + 1 + kPadPairs) * 2;  // pairs (m, m + 1) stay below this m
    // first trial: about cut x (boundaries per unit of scaled distance) boundaries on each side
    const float span = lq(n) - lq(0);
    const float per = span > 0.0f ? __fdividef((float)n, span) : 0.0f;
    int GN = (int)fminf(cut * per, (float)(n + 1)) >> 1, GP = GN;
    float r = 0.0f;
    int jb = 0;
    // ---- two adjacent slots per lane ----
    for (; n - jb > 32; jb += 64) {
        const int j = jb + 2 * lane;
        const bool actA = j < n, actB = j + 1 < n;
        const int a = actA ? j : jb;  // an idle lane shadows slot jb with zero weight
        const float4 q0 = Q[a >> 1];  // l_a, l_{a+1}, dC_a, dC_{a+1}
        const float muA = 0.5f * (q0.x + q0.y), muB = 0.5f * (q0.y + Qf[4 * ((a >> 1) + 1)]);
        const float2 Cs = *reinterpret_cast<const float2 *>(sc + a);
        const float2 Ps = *reinterpret_cast<const float2 *>(sp + a);
        const float below = muA - cut, above = (actB ? muB : muA) + cut;
        auto neg_ok = [&](int G) {
            const int m = a - 2 * G;
            return !actA || m <= 0 || lq(m - 1) < below;
        };
        auto pos_ok = [&](int G) {
            const int e = a + 2 + 2 * G;
            return !actA || e > n || lq(e) >= above;
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
        const f32x2 muA2 = pack2(muA, muA), muB2 = pack2(muB, muB);
        f32x2 accA = pack2(0.0f, 0.0f), accB = pack2(0.0f, 0.0f);
        int m = max(a - 2 * GN, -kPad2D);
#pragma unroll kPair2Unroll
        for (; m < a; m += 2) {
            const float4 q = Q[m >> 1];
            accA = pair_term<true>(q, muA2, accA);
            accB = pair_term<true>(q, muB2, accB);
        }
        accA = straddle_term(q0, muA, accA);
        accB = pair_term<true>(q0, muB2, accB);
        const int end = min(a + 2 + 2 * GP, mtop);
#pragma unroll kPair2Unroll
        for (m = a + 2; m < end; m += 2) {
            const float4 q = Q[m >> 1];
            accA = pair_term<false>(q, muA2, accA);
            accB = pair_term<false>(q, muB2, accB);
        }
        float a0, a1, b0, b1;
        unpack2(accA, a0, a1);
        unpack2(accB, b0, b1);
        r = fmaf(actA ? Ps.x : 0.0f, Cs.x + (a0 + a1), r);
        r = fmaf(actB ? Ps.y : 0.0f, Cs.y + (b0 + b1), r);
    }
    // ---- one slot per lane ----
    for (; jb < nslots; jb += 32) {
        const int j = jb + lane;
        const bool act = j < nslots;
        float mu = 0.0f, Cj = 0.0f, Pj = 0.0f;
        int mid = 0;
        if (act && j < n) {
            mu = 0.5f * (lq(j) + lq(j + 1));
            Cj = sc[j];
            Pj = sp[j];
            mid = j + 1;
        } else if (act) {  // the no-return slot: centre before l_0, every boundary above it
            mu = mu0;
            Pj = pe0;
        }
        const int nb = mid & ~1;  // pairs (m, m + 1) with m + 1 < mid end here
        const float below = mu - cut, above = mu + cut;
        auto neg_ok = [&](int G) {
            const int m = nb - 2 * G;
            return !act || m <= 0 || lq(m - 1) < below;
        };
        auto pos_ok = [&](int G) {
            const int e = nb + 2 + 2 * G;
            return !act || e > n || lq(e) >= above;
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
        const f32x2 mu2 = pack2(mu, mu);
        f32x2 acc = pack2(0.0f, 0.0f);
        int m = act ? max(nb - 2 * GN, -kPad2D) : 0;
        const int nbe = act ? nb : 0;
#pragma unroll kPairUnroll
        for (; m < nbe; m += 2) acc = pair_term<true>(Q[m >> 1], mu2, acc);
        const int end = act ? min(nb + 2 + 2 * GP, mtop) : 0;
        if (m < end) {  // the pair at nb: it straddles the centre when mid is odd, else lies above it
            const float4 q = Q[m >> 1];
            acc = (m == mid - 1) ? straddle_term(q, mu, acc) : pair_term<false>(q, mu2, acc);
            m += 2;
        }
#pragma unroll kPairUnroll
        for (; m < end; m += 2) acc = pair_term<false>(Q[m >> 1], mu2, acc);
        float a0, a1;
        unpack2(acc, a0, a1);
        r = fmaf(Pj, Cj + (a0 + a1), r);
    }
    return r;
}

// ---- the Approx-FSMI pair sum over mirrored boundary pairs -------------------------------------
//
// Interleaved boundaries for Approx-FSMI: LW[m] = (l_m, dC_m) (scaled distance, C_m - C_{m-1})
// for m in [-kPad2D, n + kPad2D], padding (l = -+3e30, dC = 0) beyond the beam. Built in place over
// sl and the scratch array after it from the top down, as build_pairs does (writing LW[m]
// overwrites l_{2m}, l_{2m+1}, which only LW[2m], LW[2m+1] read).
__device__ __forceinline__ void build_lw(float *sl, const float *sc, int n, float cs)
{
    const int lane = lane_id();
    float2 *LW = reinterpret_cast<float2 *>(sl);
    const int mend = n + 1 + kPad2D;  // boundaries 0 .. mend - 1 (those above n padding)
    for (int top = mend; top > 0; top -= 32) {
        const int m = top - 32 + lane;
        float2 v = make_float2(3.0e30f, 0.0f);
        if (m >= 0 && m <= n) v = make_float2(sl[m] * cs, sc[m] - (m > 0 ? sc[m - 1] : 0.0f));  // sc[n] = 0
        __syncwarp();
        if (m >= 0) LW[m] = v;
        __syncwarp();
    }
    LW[-1 - lane] = make_float2(-3.0e30f, 0.0f);  // kPad2D = 32 padding boundaries below 0
    __syncwarp();
}

// Approx-FSMI (eq. fsmi_approx): for first-hit slot j the band k in [klo, khi] = [j - Delta,
// j + Delta] n [0, n - 1], i.e. boundaries m in [klo, khi + 1] with C' = C on the band and 0 outside
// it. In boundary form the interior boundaries weigh dC_m, the band edges C_klo (at m = klo) and
// -C_khi (at m = khi + 1). The boundaries below the centre, j - i, and above it, j + 1 + i, are
// taken as mirrored pairs (j - i, j + 1 + i), i = 0 .. Delta, so that every pair has the signs
// (-, +), which the tail's coefficients carry, and every lane runs exactly Delta + 1 pairs: an edge
// clamped at the beam's end lands on a padding boundary (its term is 0, and dC_0 = C_0, dC_n =
// -C_{n-1} are already the clamped edges' weights), and an unclamped edge is the last pair, whose
// weights are C_{j-Delta} and -C_{j+Delta}. The no-return slot (e0) is j = -1 with centre mu0: the
// paper's band k in [1, Delta], every boundary above it. Delta beyond n changes nothing (every band
// is the whole beam), so it is capped at n; past the padding (Delta > kPad2D - 1) the indices are
// clamped to it.
template <bool CLAMP>
__device__ __forceinline__ float approx_pairs_sum(const float2 *LW, const float *sc, const float *sp, int n, bool e0,
                                                  float pe0, float mu0, int D)
{
    const int lane = lane_id();
    float r = 0.0f;
    for (int jb = e0 ? -1 : 0; jb < n; jb += 32) {
        const int j = jb + lane;
        const bool act = j < n;
        const int jj = act ? j : n - 1;  // an idle lane shadows the last slot with zero weight
        float mu, Cj, Pj;
        if (jj >= 0) {
            mu = 0.5f * (LW[jj].x + LW[jj + 1].x);
            Cj = sc[jj];
            Pj = act ? sp[jj] : 0.0f;
        } else {
            mu = mu0;
            Cj = 0.0f;
            Pj = pe0;
        }
        f32x2 acc = pack2(0.0f, 0.0f);
        int i = 0;
#pragma unroll 2
        for (; i < D; ++i) {
            const int mb = jj - i, ma = jj + 1 + i;
            const float2 b = LW[CLAMP ? max(mb, -kPad2D) : mb], a = LW[CLAMP ? min(ma, n + kPad2D) : ma];
            acc = fma2(pack2(b.y, a.y), gauss_tail2p<true, false>(pack2(mu - b.x, a.x - mu)), acc);
        }
        {  // i = D: the band edges
            const int mb = jj - D, ma = jj + 1 + D;
            const float2 b = LW[CLAMP ? max(mb, -kPad2D) : mb], a = LW[CLAMP ? min(ma, n + kPad2D) : ma];
            const float wb = mb >= 0 ? sc[mb] : 0.0f, wa = (ma >= 1 && ma <= n) ? -sc[ma - 1] : 0.0f;
            acc = fma2(pack2(wb, wa), gauss_tail2p<true, false>(pack2(mu - b.x, a.x - mu)), acc);
        }
        float a0, a1;
        unpack2(acc, a0, a1);
        r = fmaf(Pj, Cj + (a0 + a1), r);
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
        // four cells per lane in flight: all ids, then all gathers, then all stores
        constexpr int kG = 4;
        for (int i0 = lane; i0 < n; i0 += 32 * kG) {
            unsigned id[kG];
            float4 v[kG];
#pragma unroll
            for (int k = 0; k < kG; ++k) {
                const int i = i0 + 32 * k;
                id[k] = i < n ? (unsigned)((const int *)sx)[i] : ncell;
                bad |= i < n && id[k] >= ncell;  // cannot happen for a consistent traversal; never read out of bounds
            }
#pragma unroll
            for (int k = 0; k < kG; ++k) {
                v[k] = id[k] < ncell ? __ldg(gains + id[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (TRAJ && id[k] < ncell && __ldg(stamps + id[k]) < state) v[k].y = v[k].z = 0.0f;
            }
#pragma unroll
            for (int k = 0; k < kG; ++k) {
                const int i = i0 + 32 * k;
                if (i < n) {
                    sp[i] = v[k].x;
                    sc[i] = v[k].y;
                    sx[i] = v[k].z;
                }
            }
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
        const float pe0 = cell_prefixes(sp, sc, sx, n, VAR == FSMI_UNIFORM);
        if (VAR == FSMI_EXACT || VAR == kExactFullSweep) {
            const float mu0 = sl[0] * cs - 0.5f * cs;  // e_0 centre, l_1 - 1/2 (scaled)
            build_pairs(sl, sc, n, cs);
            float cut = VAR == kExactFullSweep ? __int_as_float(0x7f800000) : kTailCutDefault;
            if (VAR == FSMI_EXACT && (p.flags & FSMI_FLAG_FULL_WINDOW)) cut = kTailCut;
            I = exact_pairs_sum(reinterpret_cast<const float4 *>(sl), sc, sp, n, e0, pe0, mu0, cut);
        }
        if (VAR == FSMI_APPROX) {
            const float mu0 = sl[0] * cs - 0.5f * cs;  // e_0 centre, l_1 - 1/2 (scaled)
            build_lw(sl, sc, n, cs);
            const int D = min(p.trunc, n);
            const float2 *LW = reinterpret_cast<const float2 *>(sl);
            I = D < kPad2D ? approx_pairs_sum<false>(LW, sc, sp, n, e0, pe0, mu0, D)
                           : approx_pairs_sum<true>(LW, sc, sp, n, e0, pe0, mu0, D);
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
            int pi, bi;
            if (beam <= 0x7fffffffLL) {  // 32-bit division (the common case; the 64-bit one is far longer)
                pi = (int)((unsigned)beam / (unsigned)src.B);
                bi = (int)((unsigned)beam - (unsigned)pi * (unsigned)src.B);
            } else {
                pi = (int)(beam / src.B);
                bi = (int)(beam % src.B);
            }
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
