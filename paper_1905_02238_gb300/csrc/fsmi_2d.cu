// 2D hot path: fixed-point ray traversal, first-hit probabilities, C_k and the FSMI /
// Approx-FSMI / Uniform-FSMI pair sums, one warp per beam.
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
#include "../../include/fsmi.h"
#include "fsmi_device.cuh"
#include "dda2d.cuh"
#include "fsmi_internal.h"
#include "gauss_tail.cuh"

namespace fsmi {

// ---- pair sums ------------------------------------------------------------------------------------

// per-warp shared arrays, in units of `stride` floats: l, C, P, scratch (ids / f_emp / D / dC)
constexpr int kArrays2D = 4;
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
// Slot n is the no-return event when e0 is set (centre mu0, C_0 = 0).
template <int J>
__device__ __forceinline__ float exact_pass(const float *sl, const float *sc, const float *sp, int n, int jb,
                                            bool e0, float pe0, float mu0)
{
    const int lane = lane_id();
    float mu[J], acc[J];
    int mid[J];  // boundaries m < mid lie before the centre
#pragma unroll
    for (int t = 0; t < J; ++t) {
        const int j = jb + lane + 32 * t;
        mu[t] = (j < n) ? 0.5f * (sl[j] + sl[j + 1]) : ((j == n && e0) ? mu0 : 3.0e30f);
        mid[t] = (j < n) ? j + 1 : 0;
        acc[t] = 0.0f;
    }
    float cprev = 0.0f;
    for (int m = 0; m <= n; ++m) {
        const float lm = sl[m];
        const float cm = sc[m];  // sc[n] = 0 (C_{n+1})
        const float dc = cm - cprev;
        cprev = cm;
#pragma unroll
        for (int t = 0; t < J; ++t) acc[t] = fmaf(m < mid[t] ? -dc : dc, gauss_tail(lm - mu[t]), acc[t]);
    }
    float r = 0.0f;
#pragma unroll
    for (int t = 0; t < J; ++t) {
        const int j = jb + lane + 32 * t;
        if (j < n)
            r = fmaf(sp[j], sc[j] + acc[t], r);
        else if (j == n && e0)
            r = fmaf(pe0, acc[t], r);
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

__device__ __forceinline__ int lower_bound_f(const float *a, int n, float x)
{
    int lo = 0, len = n;
    while (len > 0) {
        const int half = len >> 1;
        if (a[lo + half] < x) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

// Boundary terms m in [a, b) of one first-hit cell, added in increasing m to acc: on the lower
// side (NEG, boundaries before the centre) the term is -dC_m T(mu - l_m), above it +dC_m T(l_m - mu).
// Aligned pairs of boundaries go through the packed tail; results equal the scalar path bit for bit.
#ifndef FSMI_PAIR_UNROLL
#define FSMI_PAIR_UNROLL 4
#endif
constexpr int kPairUnroll = FSMI_PAIR_UNROLL;  // boundary pairs in flight per lane, exact window loop

template <bool NEG>
__device__ __forceinline__ float side_terms(const float *sl, const float *sdc, int a, int b, float mu, float acc)
{
    int m = a;
    if (m < b && (m & 1)) {
        const float d = NEG ? mu - sl[m] : sl[m] - mu;
        acc = fmaf(NEG ? -sdc[m] : sdc[m], gauss_tail(d), acc);
        ++m;
    }
    const f32x2 mu2 = pack2(mu, mu);
#pragma unroll kPairUnroll
    for (; m + 1 < b; m += 2) {
        const f32x2 L = *reinterpret_cast<const f32x2 *>(sl + m);
        const float2 dc = *reinterpret_cast<const float2 *>(sdc + m);
        float T0, T1;
        gauss_tail2(NEG ? sub2(mu2, L) : sub2(L, mu2), T0, T1);
        acc = fmaf(NEG ? -dc.x : dc.x, T0, acc);
        acc = fmaf(NEG ? -dc.y : dc.y, T1, acc);
    }
    if (m < b) {
        const float d = NEG ? mu - sl[m] : sl[m] - mu;
        acc = fmaf(NEG ? -sdc[m] : sdc[m], gauss_tail(d), acc);
    }
    return acc;
}

// Exact pair sum over the boundaries whose tail term can be non-zero: for slot j only
// m with |l_m - mu_j| < kTailCut (scaled) are visited, in increasing m, so every non-zero term
// of the full sweep is added in the same order and the FP32 result is the same bit for bit.
// sdc[m] = C_m - C_{m-1} for m = 0..n.
__device__ __forceinline__ float exact_window_sum(const float *sl, const float *sdc, const float *sc,
                                                  const float *sp, int n, bool e0, float pe0, float mu0)
{
    const int nslots = n + (e0 ? 1 : 0);
    float r = 0.0f;
    for (int j = lane_id(); j < nslots; j += 32) {
        float mu, Cj, Pj;
        int mid;
        if (j < n) {
            mu = 0.5f * (sl[j] + sl[j + 1]);
            Cj = sc[j];
            Pj = sp[j];
            mid = j + 1;
        } else {
            mu = mu0;
            Cj = 0.0f;
            Pj = pe0;
            mid = 0;
        }
        const int lo = lower_bound_f(sl, n + 1, mu - kTailCut);
        const int hi = lower_bound_f(sl, n + 1, mu + kTailCut);
        float acc = side_terms<true>(sl, sdc, lo, min(max(mid, lo), hi), mu, 0.0f);
        acc = side_terms<false>(sl, sdc, max(mid, lo), hi, mu, acc);
        r = fmaf(Pj, Cj + acc, r);
    }
    return r;
}

// Approx-FSMI: for slot j the band k in [klo, khi] = [j - Delta, j + Delta] n [0, n-1] (0-based),
// i.e. boundaries m in [klo, khi + 1] with C' = C on the band and 0 outside it.
__device__ __forceinline__ float approx_sum(const float *sl, const float *sc, const float *sp, int n, bool e0,
                                            float pe0, float mu0, int D)
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
        for (int m = klo; m <= khi + 1; ++m) {
            const float cm = (m <= khi) ? sc[m] : 0.0f;
            const float cm1 = (m > klo) ? sc[m - 1] : 0.0f;
            const float dc = cm - cm1;
            acc = fmaf(m < mid ? -dc : dc, gauss_tail(sl[m] - mu), acc);
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
#define FSMI_MIN_BLOCKS_2D 1  // minimum resident blocks per SM requested from the register allocator
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

// One beam: traversal (or explicit cells), gains, prefixes, the variant's pair sum, store.
template <int VAR, int SRC>
__device__ __forceinline__ void eval_beam(const Src2D &src, const DevParams &p, long long beam, float *sl, float *sc,
                                          float *sp, float *sx, float *__restrict__ out, int *status)
{
    const int lane = lane_id();
    const bool e0 = p.e0 != 0;
    const float cs = p.inv_s2 * (float)kSqrtLog2e;  // distance -> tail variable
    int n;
    if (SRC != kSrcBeams) {
        const int32_t *pose;
        int ux, uy;
        int state = 0;                   // kSrcTraj: state index within the trajectory
        const int32_t *stamps = nullptr;  // kSrcTraj: the trajectory's visit stamps
        long long rfix = p.rfix;
        float rend = p.rend;
        int cap = p.nmax;
        if (SRC == kSrcMap || SRC == kSrcTraj) {
            const int pi = (int)(beam / src.B), bi = (int)(beam % src.B);
            pose = src.poses + 4 * (size_t)pi;
            ux = src.dirs[2 * bi];
            uy = src.dirs[2 * bi + 1];
            if (SRC == kSrcTraj) {
                const int t = traj_of(src.traj_off, src.T, pi);
                if (t < 0) {  // pose not covered by the trajectory offsets
                    if (lane == 0) {
                        out[beam] = __int_as_float(0x7fc00000);
                        set_status(status, FSMI_STATUS_BAD_BEAM);
                    }
                    return;
                }
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
            if (!ok) {  // malformed descriptor: never index with it
                if (lane == 0) {
                    out[beam] = __int_as_float(0x7fc00000);
                    set_status(status, FSMI_STATUS_BAD_BEAM);
                }
                return;
            }
            pose = src.poses + 4 * (size_t)pi;
            ux = src.dirs[2 * bi];
            uy = src.dirs[2 * bi + 1];
        }
        int dx, dy;
        beam_dir(pose, ux, uy, dx, dy);
        n = dda_warp(src.W, src.H, pose[0], pose[1], dx, dy, rfix, rend, cap, (int *)sx, sl);
        if (n < 0) {
            if (lane == 0) {
                out[beam] = __int_as_float(0x7fc00000);
                set_status(status, FSMI_STATUS_BEAM_OVERFLOW);
            }
            __syncwarp();
            return;
        }
        const unsigned ncell = (unsigned)src.W * (unsigned)src.H;
        bool bad = false;
        if (src.gains) {
            for (int i = lane; i < n; i += 32) {
                const unsigned id = (unsigned)((const int *)sx)[i];
                bad |= id >= ncell;  // cannot happen for a consistent traversal; never read out of bounds
                float4 v = id < ncell ? __ldg(src.gains + id) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (SRC == kSrcTraj && id < ncell && __ldg(stamps + id) < state) v.y = v.z = 0.0f;
                sp[i] = v.x;
                sc[i] = v.y;
                sx[i] = v.z;
            }
        } else {
            for (int i = lane; i < n; i += 32) {
                const unsigned id = (unsigned)((const int *)sx)[i];
                bad |= id >= ncell;
                const float o = id < ncell ? __ldg(src.map + id) : 0.0f;
                // a cell already counted by an earlier state of the trajectory (Section 2.4) still
                // stops the beam with probability o but adds no information
                const bool counted = SRC == kSrcTraj && id < ncell && __ldg(stamps + id) < state;
                sp[i] = o;
                sc[i] = counted ? 0.0f : cell_gain(p.docc, o);
                sx[i] = counted ? 0.0f : cell_gain(p.demp, o);
            }
        }
        if (__any_sync(kFull, bad) && lane == 0) set_status(status, FSMI_STATUS_INTERNAL);
    } else {
        const int base = src.off[beam];
        n = src.off[beam + 1] - base;
        if (n < 0 || n > p.nmax) {
            if (lane == 0) {
                out[beam] = __int_as_float(0x7fc00000);
                set_status(status, FSMI_STATUS_BAD_BEAM);
            }
            return;
        }
        for (int i = lane; i < n; i += 32) {
            const float o = __ldg(src.o + base + i);
            sl[i] = __ldg(src.l + base + i);
            sp[i] = o;
            sc[i] = cell_gain(p.docc, o);
            sx[i] = cell_gain(p.demp, o);
        }
        if (lane == 0) sl[n] = __ldg(src.lend + beam);
    }
    __syncwarp();
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
            __syncwarp();
            I = exact_window_sum(sl, sx, sc, sp, n, e0, pe0, mu0);
        }
        if (VAR == FSMI_APPROX) I = approx_sum(sl, sc, sp, n, e0, pe0, mu0, p.trunc);
        if (VAR == FSMI_UNIFORM) I = uniform_sum(sx, sp, n, e0, pe0, p.H, p.inv_2h1);
        I = warp_sum(I);
    }
    if (lane == 0) out[beam] = I;
    __syncwarp();
}

// Persistent kernel: each warp evaluates beams one at a time, either in a static grid-stride
// order or, with a work queue, taking `chunk` consecutive beams per atomic grab (balances beams
// of very different lengths). The queue counter must be zero at launch.
template <int VAR, int SRC>
__global__ void __launch_bounds__(kMaxWarps * 32, FSMI_MIN_BLOCKS_2D)
    k_eval_2d(Src2D src, DevParams p, long long nbeams, int stride, float *__restrict__ out, int *status,
              unsigned long long *queue, int chunk)
{
    extern __shared__ float smem[];
    const int lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float *sl = smem + (size_t)warp * kArrays2D * stride;
    float *sc = sl + stride;
    float *sp = sc + stride;
    float *sx = sp + stride;
    for_each_item(nbeams, queue, chunk,
                  [&](long long beam) { eval_beam<VAR, SRC>(src, p, beam, sl, sc, sp, sx, out, status); });
}

__global__ void __launch_bounds__(128)
    k_trace_2d(int W, int H, const int32_t *__restrict__ poses, const int32_t *__restrict__ dirs, int B,
               long long nbeams, long long rfix, float rend, int cap, int32_t *__restrict__ cells,
               float *__restrict__ l, int32_t *__restrict__ nout)
{
    const int warp = threadIdx.x >> 5;
    for (long long beam = (long long)blockIdx.x * 4 + warp; beam < nbeams; beam += (long long)gridDim.x * 4) {
        const int pi = (int)(beam / B), bi = (int)(beam % B);
        const int32_t *pose = poses + 4 * (size_t)pi;
        int dx, dy;
        beam_dir(pose, dirs[2 * bi], dirs[2 * bi + 1], dx, dy);
        const int n = dda_warp(W, H, pose[0], pose[1], dx, dy, rfix, rend, cap, cells + beam * cap,
                               l + beam * (cap + 1));
        if (lane_id() == 0) nout[beam] = n;
    }
}

// Per-cell gains of the whole map: (o, f(delta_occ, r), f(delta_emp, r), 0), the same values the
// beam kernel would compute at each visit.
__global__ void k_map_gains(const float *__restrict__ map, long long ncell, float docc, float demp,
                            float4 *__restrict__ gains)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += (long long)gridDim.x * blockDim.x) {
        const float o = __ldg(map + i);
        gains[i] = make_float4(o, cell_gain(docc, o), cell_gain(demp, o), 0.0f);
    }
}

// Scaled Gaussian tail over an array (exposed for testing the numerical core).
__global__ void k_gauss_tail(const float *__restrict__ s, float *__restrict__ out, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = gauss_tail(s[i]);
}


template <int VAR, int SRC>
static cudaError_t launch_variant(const Src2D &src, const DevParams &p, long long nbeams, float *out, int *status,
                                  unsigned long long *queue, cudaStream_t s)
{
    const Schedule &sc = current_schedule(FSMI_KIND_2D);
    const int stride = ((p.nmax + 2) + 3) & ~3;
    const size_t per_warp = (size_t)kArrays2D * stride * sizeof(float);
    const int wpb = fit_warps(sc.warps_per_block, per_warp, 0);
    const size_t smem = (size_t)wpb * per_warp;
    auto kern = k_eval_2d<VAR, SRC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (sc.blocks_per_sm > 0 && sc.blocks_per_sm < occ) occ = sc.blocks_per_sm;
    long long want = (nbeams + wpb - 1) / wpb;
    long long grid = (long long)sm_count() * occ;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    if (queue) {
        e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)grid, wpb * 32, smem, s>>>(src, p, nbeams, stride, out, status, queue,
                                                 sc.queue_chunk > 0 ? sc.queue_chunk : 1);
    return cudaGetLastError();
}

template <int SRC>
static cudaError_t dispatch(const Src2D &src, const DevParams &p, long long nbeams, float *out, int *status,
                            unsigned long long *queue, cudaStream_t s)
{
    if (nbeams <= 0) return cudaSuccess;
    switch (p.variant) {
        case FSMI_EXACT:
            if (p.flags & FSMI_FLAG_FULL_SWEEP) return launch_variant<kExactFullSweep, SRC>(src, p, nbeams, out, status, queue, s);
            return launch_variant<FSMI_EXACT, SRC>(src, p, nbeams, out, status, queue, s);
        case FSMI_APPROX: return launch_variant<FSMI_APPROX, SRC>(src, p, nbeams, out, status, queue, s);
        default: return launch_variant<FSMI_UNIFORM, SRC>(src, p, nbeams, out, status, queue, s);
    }
}

static cudaError_t map_gains(const float *map, int W, int H, const DevParams &p, float4 *gains, cudaStream_t s)
{
    const long long ncell = (long long)W * H;
    long long grid = (ncell + 255) / 256;
    const long long gmax = (long long)sm_count() * 16;
    if (grid > gmax) grid = gmax;
    k_map_gains<<<(unsigned)grid, 256, 0, s>>>(map, ncell, p.docc, p.demp, gains);
    return cudaGetLastError();
}

cudaError_t launch_eval_2d(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                           const DevParams &p, float *out, float4 *gains, unsigned long long *queue, int *status,
                           cudaStream_t s)
{
    if (gains) {
        cudaError_t e = map_gains(map, W, H, p, gains, s);
        if (e != cudaSuccess) return e;
    }
    Src2D src{map, W, H, poses, P, dirs, B, gains, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, 0, nullptr};
    return dispatch<kSrcMap>(src, p, (long long)P * B, out, status, queue, s);
}

cudaError_t launch_eval_2d_sets(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs,
                                int B, const fsmi_set_2d *sets, int nsets, long long nbeams, const DevParams &p, float *out,
                                float4 *gains, unsigned long long *queue, int *status, cudaStream_t s)
{
    if (gains) {
        cudaError_t e = map_gains(map, W, H, p, gains, s);
        if (e != cudaSuccess) return e;
    }
    Src2D src{map, W, H, poses, P, dirs, B, gains, nullptr, nullptr, nullptr, nullptr, sets, nsets, nullptr, 0, nullptr};
    return dispatch<kSrcSets>(src, p, nbeams, out, status, queue, s);
}

cudaError_t launch_eval_2d_traj(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *traj_off,
                                int T, const int32_t *stamp, const int32_t *dirs, int B, const DevParams &p, float *out,
                                float4 *gains, unsigned long long *queue, int *status, cudaStream_t s)
{
    if (gains) {
        cudaError_t e = map_gains(map, W, H, p, gains, s);
        if (e != cudaSuccess) return e;
    }
    Src2D src{map, W, H, poses, P, dirs, B, gains, nullptr, nullptr, nullptr, nullptr, nullptr, 0, traj_off, T, stamp};
    return dispatch<kSrcTraj>(src, p, (long long)P * B, out, status, queue, s);
}

cudaError_t launch_eval_beams(const int32_t *off, const float *o, const float *l, const float *lend, int nbeams,
                              const DevParams &p, float *out, unsigned long long *queue, int *status, cudaStream_t s)
{
    Src2D src{nullptr, 0, 0, nullptr, 0, nullptr, 0, nullptr, off, o, l, lend, nullptr, 0, nullptr, 0, nullptr};
    return dispatch<kSrcBeams>(src, p, nbeams, out, status, queue, s);
}

// Loads every 2D kernel on the current device (a kernel's first use loads it lazily).
template <int SRC>
static cudaError_t prepare_src()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_eval_2d<FSMI_EXACT, SRC>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_2d<kExactFullSweep, SRC>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_2d<FSMI_APPROX, SRC>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_2d<FSMI_UNIFORM, SRC>);
    return e;
}

cudaError_t prepare_2d()
{
    cudaError_t e = prepare_src<kSrcMap>();
    if (e == cudaSuccess) e = prepare_src<kSrcBeams>();
    if (e == cudaSuccess) e = prepare_src<kSrcSets>();
    if (e == cudaSuccess) e = prepare_src<kSrcTraj>();
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_map_gains);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_trace_2d);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_gauss_tail);
    return e;
}

cudaError_t launch_trace_2d(int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B, long long rfix,
                            float rend, int cap, int32_t *cells, float *l, int32_t *n, cudaStream_t s)
{
    const long long nb = (long long)P * B;
    if (nb <= 0) return cudaSuccess;
    long long grid = (nb + 3) / 4;
    const long long gmax = (long long)sm_count() * 16;
    if (grid > gmax) grid = gmax;
    k_trace_2d<<<(unsigned)grid, 128, 0, s>>>(W, H, poses, dirs, B, nb, rfix, rend, cap, cells, l, n);
    return cudaGetLastError();
}

cudaError_t launch_gauss_tail(const float *sv, float *out, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long grid = (n + 255) / 256;
    const long long gmax = (long long)sm_count() * 8;
    if (grid > gmax) grid = gmax;
    k_gauss_tail<<<(unsigned)grid, 256, 0, s>>>(sv, out, n);
    return cudaGetLastError();
}

}  // namespace fsmi
