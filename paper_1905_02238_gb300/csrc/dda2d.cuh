// Fixed-point 2D ray traversal shared by the evaluation, visit-stamp and map-update kernels: the
// cells a beam crosses (Section 2.2 lists them in ascending distance) with their entry distances.
#pragma once

#include <stdint.h>

#include "fsmi_device.cuh"

namespace fsmi {

// Beam direction: the sensor-frame unit vector u rotated by the pose's (cos, sin), rounded half
// up: d = floor((Rot u + 2^29) / 2^30). Arithmetic right shift is a floor division by 2^30.
__device__ __forceinline__ void beam_dir(const int32_t *pose, int32_t ux, int32_t uy, int &dx, int &dy)
{
    const long long c = pose[2], s = pose[3];
    dx = (int)((c * ux - s * uy + (1LL << 29)) >> 30);
    dy = (int)((s * ux + c * uy + (1LL << 29)) >> 30);
}

// ---- traversal ----------------------------------------------------------------------------------
//
// The beam is o + lambda * d / 2^30 (o in Q16 cell units, d in Q30); lambda is its distance. Cells
// change at x crossings lambda_x(a) = (nx0 + a 2^16) 2^14 / |dx| and y crossings likewise, with
// nx0, ny0 the Q16 distances from o to the far side of the first cell (the cell entered by
// o + eps d). Crossings are ordered by exact int64 comparison; coinciding crossings are one
// diagonal step. A cell is entered while its entry lambda < R and it lies inside the grid.
//
// Parallel form: along the major axis M (|d_M| >= |d_m|) consecutive M-crossings split the beam
// into intervals [lambda_M(k), lambda_M(k+1)), k = -1, 0, 1, ... (lambda_M(-1) = 0). Minor
// crossings are at least as far apart as major ones, so each interval holds the cell entered at
// its start plus at most one cell entered at a minor crossing strictly inside it. Lane L walks a
// contiguous block of intervals k0..k1; its starting minor coordinate is the number of minor
// crossings at or before lambda_M(k0) (one integer division). Its cell count, unless the beam
// ends inside the block, is (k1 - k0 + 1) + (minor crossings in (lambda_M(k0), lambda_M(k1+1)])
// minus the crossings among those that coincide with a major crossing (diagonal steps, which
// enter one cell, not two). The lanes write their cells at offsets from a warp scan of that count
// taken without the coincidences, and count the coincidences as they walk; if a lane before the
// one where the beam ends met any, the offsets were too large and the lanes walk again at the
// exact offsets (beams along a lattice diagonal through cell centres; rare otherwise). The first
// lane that meets the range limit or the grid boundary ends the beam.

struct Geo {
    int sM, sm, cM0, cm0, dimM, dimm, xmaj, W;
    unsigned nM0, nm0;  // Q16 distances to the first major / minor boundary (< 2^31 + 2^16 with k)
    unsigned aM, am;    // |d| along the major / minor axis (Q30, <= 2^31)
    unsigned LM, Lm;    // crossing numerators below these have entry distance < R
    float rM, rm, R;
};

__device__ __forceinline__ unsigned long long mulw(unsigned a, unsigned b) { return (unsigned long long)a * b; }

// Number of minor crossings at or before the major crossing k: #{i >= 0 : nm(i) aM <= nM(k) am}
// = floor((nM(k) am - nm0 aM) / (2^16 aM)) + 1 when that numerator is >= 0. The quotient (< 2^11
// for ranges up to 1024 cells) is estimated in FP32 and corrected exactly in integers.
__device__ __forceinline__ int minor_before(const Geo &g, int k)
{
    if (g.am == 0 || k < 0) return 0;
    const long long num = (long long)mulw(g.nM0 + (unsigned)k * 65536u, g.am) - (long long)mulw(g.nm0, g.aM);
    if (num < 0) return 0;
    const long long hi = num >> 16;  // floor(num / 2^16); floor(hi / aM) = floor(num / (2^16 aM))
    long long q = (long long)((float)hi * (1.0f / (float)g.aM));
    q -= (q * (long long)g.aM > hi);
    q -= (q * (long long)g.aM > hi);
    q += ((q + 1) * (long long)g.aM <= hi);
    q += ((q + 1) * (long long)g.aM <= hi);
    return (int)q + 1;
}

// Walks intervals k0..k1 from minor crossing i0 = minor_before(k0), writing (WRITE) its cells
// from index `base`; cnt = cells entered, ties = minor crossings that coincided with a major one
// (diagonal steps) before the walk ended. CHECK: skip writes at indices >= cap (not needed when
// every index the walk can reach is below cap). The current cell's id advances with its
// coordinates (by stepM per major step, stepm per minor step) rather than being recomputed.
template <bool WRITE, bool CHECK = true>
__device__ __forceinline__ void walk(const Geo &g, int k0, int k1, int i0, int base, int cap, int *ids, float *l,
                                     int &cnt, int &ties, bool &ended, float &endl, bool &by_range)
{
    int cM = g.cM0 + g.sM * (k0 + 1);
    int i = i0;
    int cm = g.cm0 + g.sm * i;
    const int stepM = g.xmaj ? g.sM : g.sM * g.W, stepm = g.xmaj ? g.sm * g.W : g.sm;
    int id = g.xmaj ? (cm * g.W + cM) : (cM * g.W + cm);
    int *ip = ids + base;
    float *lp = l + base;
    cnt = 0;
    ties = 0;
    ended = false;
    endl = 0.0f;
    by_range = false;
#define FSMI_EMIT(lam_)                                                              \
    do {                                                                             \
        if (WRITE && (!CHECK || base + cnt < cap)) {                                 \
            *ip = id;                                                                \
            *lp = (lam_);                                                            \
        }                                                                            \
        ++ip;                                                                        \
        ++lp;                                                                        \
        ++cnt;                                                                       \
    } while (0)
    // crossings are compared as nm(i) aM against nM(k + 1) am; both products advance by constant
    // steps (aM 2^16 per minor crossing, am 2^16 per interval), so the loop multiplies nothing
    unsigned nMn = g.nM0 + (unsigned)(k0 + 1) * 65536u;  // next major crossing
    unsigned nmi = g.nm0 + (unsigned)i * 65536u;         // next minor crossing
    unsigned long long pm = mulw(nmi, g.aM), pM = mulw(nMn, g.am);
    const unsigned long long dm = (unsigned long long)g.aM << 16, dM = (unsigned long long)g.am << 16;
    for (int k = k0; k <= k1; ++k, nMn += 65536u, pM += dM) {
        FSMI_EMIT(k < 0 ? 0.0f : (float)(nMn - 65536u) * g.rM);
        const bool minor = g.am && pm < pM;  // a minor crossing inside the interval
        if (minor && (nmi >= g.Lm || (unsigned)(cm + g.sm) >= (unsigned)g.dimm)) {  // the beam ends there
            ended = true;
            by_range = nmi >= g.Lm;
            endl = by_range ? g.R : (float)nmi * g.rm;
            break;
        }
        if (minor) {  // no branch inside: the lanes stay together whichever of them cross
            cm += g.sm;
            id += stepm;
            FSMI_EMIT((float)nmi * g.rm);
            ++i;
            nmi += 65536u;
            pm += dm;
        }
        if (nMn >= g.LM) {
            ended = true;
            endl = g.R;
            by_range = true;
            break;
        }
        const bool tie = g.am && pm == pM;
        cM += g.sM;
        id += stepM;
        if (tie) {
            cm += g.sm;
            id += stepm;
            ++i;
            nmi += 65536u;
            pm += dm;
            ++ties;
        }
        if ((unsigned)cM >= (unsigned)g.dimM || (unsigned)cm >= (unsigned)g.dimm) {
            ended = true;
            endl = (float)nMn * g.rM;
            break;
        }
    }
#undef FSMI_EMIT
}

// All 32 lanes call this. Writes ids[0..n-1] (cell y*W + x) and l[0..n] (entry distances, then
// the end distance) and returns n; returns -1 (writing nothing) if the beam has more than cap
// cells. rend = R as float. *end_by_range (optional) = whether the beam ended at the range limit
// inside the grid (false when it left the grid first or crossed no cell).
static __device__ int dda_warp(int W, int H, int ox, int oy, int dx, int dy, long long rfix, float rend, int cap, int *ids,
                               float *l, bool *end_by_range = nullptr)
{
    const int lane = lane_id();
    if (end_by_range) *end_by_range = false;
    if ((dx | dy) == 0) return 0;
    int cx = ox >> 16, cy = oy >> 16;
    if (dx < 0 && (ox & 0xFFFF) == 0) --cx;
    if (dy < 0 && (oy & 0xFFFF) == 0) --cy;
    if ((unsigned)cx >= (unsigned)W || (unsigned)cy >= (unsigned)H) return 0;
    const unsigned adx = dx < 0 ? 0u - (unsigned)dx : (unsigned)dx, ady = dy < 0 ? 0u - (unsigned)dy : (unsigned)dy;
    Geo g;
    g.xmaj = adx >= ady;
    g.W = W;
    g.aM = g.xmaj ? adx : ady;
    g.am = g.xmaj ? ady : adx;
    const int dM = g.xmaj ? dx : dy, dm = g.xmaj ? dy : dx;
    g.sM = dM > 0 ? 1 : -1;
    g.sm = dm > 0 ? 1 : -1;
    g.cM0 = g.xmaj ? cx : cy;
    g.cm0 = g.xmaj ? cy : cx;
    g.dimM = g.xmaj ? W : H;
    g.dimm = g.xmaj ? H : W;
    const long long oM = g.xmaj ? ox : oy, om = g.xmaj ? oy : ox;
    g.nM0 = (unsigned)(g.sM > 0 ? ((long long)(g.cM0 + 1) << 16) - oM : oM - ((long long)g.cM0 << 16));
    g.nm0 = g.am == 0 ? 0u
                      : (unsigned)(g.sm > 0 ? ((long long)(g.cm0 + 1) << 16) - om : om - ((long long)g.cm0 << 16));
    // crossing numerators below these limits have entry lambda < R:
    //   num * 2^30 < rfix * a  <=>  num < floor((rfix * a - 1) / 2^30) + 1
    g.LM = (unsigned)((((unsigned long long)rfix * g.aM - 1) >> 30) + 1);
    g.Lm = g.am ? (unsigned)((((unsigned long long)rfix * g.am - 1) >> 30) + 1) : 0u;
    g.rM = __fdividef(16384.0f, (float)g.aM);  // distances need not be correctly rounded (< 2 ulp)
    g.rm = g.am ? __fdividef(16384.0f, (float)g.am) : 0.0f;
    g.R = rend;
    // major crossings that stay in range and inside the grid along M
    const long long KR = g.LM > g.nM0 ? ((long long)g.LM - g.nM0 + 65535) >> 16 : 0;
    const long long KG = g.sM > 0 ? (g.dimM - 1 - g.cM0) : g.cM0;
    const int K = (int)(KR < KG ? KR : KG);
    const int NI = K + 1;  // intervals k = -1 .. K-1
    const int q = (NI + 31) >> 5;
    const int k0 = -1 + lane * q;
    const int k1 = min(K - 1, k0 + q - 1);
    int cnt = 0, ties = 0;
    bool ended = false, rng = false;
    float endl = 0.0f;
    // minor crossings before each lane's first interval: lane L's block ends where lane L + 1's
    // begins, so one count per lane (at the end of its block) serves both
    const int iend = k0 <= k1 ? minor_before(g, k1 + 1) : 0;
    int i0 = __shfl_up_sync(kFull, iend, 1);
    if (lane == 0) i0 = 0;  // k0 = -1: no minor crossing before the start
    int pred = 0;
    if (k0 <= k1) pred = (k1 - k0 + 1) + iend - i0;
    const int pinc = warp_incl_add_int(pred);
    // a lane writes at most its predicted count from its offset, so every index stays below the
    // predicted total: within cap, the writes need no check
    const bool fits = __shfl_sync(kFull, pinc, 31) <= cap;
    if (k0 <= k1) {
        if (fits)
            walk<true, false>(g, k0, k1, i0, pinc - pred, cap, ids, l, cnt, ties, ended, endl, rng);
        else
            walk<true, true>(g, k0, k1, i0, pinc - pred, cap, ids, l, cnt, ties, ended, endl, rng);
    }
    const unsigned eb = __ballot_sync(kFull, ended);
    const int first = eb ? __ffs(eb) - 1 : 31;
    const float lend = __shfl_sync(kFull, endl, first);
    const unsigned rb = __ballot_sync(kFull, rng);
    if (end_by_range) *end_by_range = (rb >> first) & 1u;
    int n;
    if (__any_sync(kFull, lane < first && ties > 0)) {
        // offsets of lanes after a diagonal step were too large: count exactly, place the cells again
        const int c = lane <= first ? cnt : 0;
        const int inc = warp_incl_add_int(c);
        n = __shfl_sync(kFull, inc, 31);
        if (n > cap) return -1;
        __syncwarp();
        if (lane <= first && k0 <= k1) walk<true, false>(g, k0, k1, i0, inc - c, cap, ids, l, cnt, ties, ended, endl, rng);
    } else {
        // every lane before the first that ended walked its whole block without a diagonal step,
        // so its predicted count was exact: n = that lane's offset + its count
        n = __shfl_sync(kFull, pinc - pred + cnt, first);
        if (n > cap) return -1;
    }
    if (lane == 0) l[n] = lend;
    __syncwarp();
    return n;
}

}  // namespace fsmi
