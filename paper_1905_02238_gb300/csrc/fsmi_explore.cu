// The exploration loop around the per-beam mutual information:
//  - trajectory aggregation (Section 2.4): the MI of a discretised trajectory is the sum over its
//    states of the scan MI, where a cell that already contributed at an earlier state is marked
//    and adds nothing later. Marks are visit stamps: stamp[t][cell] = the first state of
//    trajectory t whose beams cross the cell (atomicMin over all of its beams), so a beam of state
//    s counts a cell only when stamp >= s. Sums are done in a fixed order (one warp per segment).
//  - the choice among candidate trajectories by MI per travel distance (Sections 2.4 and 5.2).
//  - the Bayesian occupancy update of eq. (1) (Section 2.1) with the inverse sensor model of Section 2.2:
//    posterior odds = prior odds x delta_occ for the cell where the measured range ends and
//    x delta_emp for every cell the beam crossed before it (x 1 beyond). Odds updates commute,
//    so a batch of beams is applied as per-cell counts: logit' = logit + a ln delta_occ + b ln delta_emp.
#include <float.h>

#include "../../include/fsmi.h"
#include "dda2d.cuh"
#include "fsmi_device.cuh"
#include "fsmi_internal.h"

namespace fsmi {

namespace {

constexpr int kWarpsExplore = 4;

// trajectory of pose p: t with off[t] <= p < off[t+1], or -1
__device__ __forceinline__ int segment_of(const int32_t *off, int T, int p)
{
    int lo = 0, len = T + 1;
    while (len > 0) {
        const int half = len >> 1;
        if (__ldg(off + lo + half) <= p) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    const int t = lo - 1;
    return (t >= 0 && t < T && p < __ldg(off + t + 1)) ? t : -1;
}

__global__ void __launch_bounds__(kWarpsExplore * 32)
    k_traj_stamps(int W, int H, const int32_t *__restrict__ poses, int P, const int32_t *__restrict__ traj_off, int T,
                  const int32_t *__restrict__ dirs, int B, long long rfix, float rend, int cap, int stride,
                  int32_t *__restrict__ stamp, int *status)
{
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    float *sl = smem + (size_t)warp * 2 * stride;
    int *ids = (int *)(sl + stride);
    const long long nbeams = (long long)P * B;
    const unsigned ncell = (unsigned)W * (unsigned)H;
    for (long long beam = (long long)blockIdx.x * kWarpsExplore + warp; beam < nbeams;
         beam += (long long)gridDim.x * kWarpsExplore) {
        const int pi = (int)(beam / B), bi = (int)(beam % B);
        const int t = segment_of(traj_off, T, pi);
        if (t < 0) {
            if (lane == 0) set_status(status, FSMI_STATUS_BAD_BEAM);
            continue;
        }
        const int s = pi - __ldg(traj_off + t);
        const int32_t *pose = poses + 4 * (size_t)pi;
        int dx, dy;
        beam_dir(pose, dirs[2 * bi], dirs[2 * bi + 1], dx, dy);
        const int n = dda_warp(W, H, pose[0], pose[1], dx, dy, rfix, rend, cap, ids, sl);
        if (n < 0) {
            if (lane == 0) set_status(status, FSMI_STATUS_BEAM_OVERFLOW);
            continue;
        }
        int32_t *row = stamp + (size_t)t * ncell;
        for (int i = lane; i < n; i += 32) {
            const unsigned id = (unsigned)ids[i];
            if (id < ncell) atomicMin(row + id, s);
        }
        __syncwarp();
    }
}

// out[r] = sum of v[r*cols .. r*cols+cols-1], one warp per row, fixed order
__global__ void k_row_sums(const float *__restrict__ v, long long rows, int cols, float *__restrict__ out)
{
    const int lane = lane_id();
    const long long wpb = blockDim.x >> 5;
    for (long long r = blockIdx.x * wpb + (threadIdx.x >> 5); r < rows; r += (long long)gridDim.x * wpb) {
        const float *x = v + r * cols;
        float a = 0.0f;
        for (int i = lane; i < cols; i += 32) a += x[i];
        a = warp_sum(a);
        if (lane == 0) out[r] = a;
    }
}

// segment [off[t], off[t+1]) clamped to [0, nv): malformed offsets never index out of bounds
__device__ __forceinline__ void segment(const int32_t *off, int t, int nv, int &a, int &b)
{
    a = min(max(off[t], 0), nv);
    b = min(max(off[t + 1], a), nv);
}

// out[t] = sum of v[off[t] .. off[t+1]-1], one warp per segment, fixed order
__global__ void k_csr_sums(const float *__restrict__ v, int nv, const int32_t *__restrict__ off, int nseg,
                           float *__restrict__ out)
{
    const int lane = lane_id();
    const int wpb = blockDim.x >> 5;
    for (int t = blockIdx.x * wpb + (threadIdx.x >> 5); t < nseg; t += gridDim.x * wpb) {
        int a, b;
        segment(off, t, nv, a, b);
        float acc = 0.0f;
        for (int i = a + lane; i < b; i += 32) acc += v[i];
        acc = warp_sum(acc);
        if (lane == 0) out[t] = acc;
    }
}

// Travel distance of trajectory t: the sum of the straight segments between consecutive states
// (cells), at least one cell so that a single-state trajectory has a finite ratio.
__device__ float path_length(const int32_t *poses, int a, int b)
{
    double len = 0.0;
    for (int s = a + 1; s < b; ++s) {
        const double dx = (double)(poses[4 * s] - poses[4 * (s - 1)]) * (1.0 / 65536.0);
        const double dy = (double)(poses[4 * s + 1] - poses[4 * (s - 1) + 1]) * (1.0 / 65536.0);
        len += sqrt(dx * dx + dy * dy);
    }
    return (float)fmax(len, 1.0);
}

// ratio[t] = traj_mi[t] / path_length(t); *best = argmax (lowest index among equal ratios; -1 if T
// has no trajectory with a finite ratio). One block.
__global__ void __launch_bounds__(1024)
    k_best_trajectory(const float *__restrict__ traj_mi, const int32_t *__restrict__ poses, int P,
                      const int32_t *__restrict__ traj_off, int T, float *__restrict__ ratio, int32_t *best)
{
    __shared__ float sv[32];
    __shared__ int si[32];
    float bv = -FLT_MAX;
    int bi = -1;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int a, b;
        segment(traj_off, t, P, a, b);
        const float r = traj_mi[t] / path_length(poses, a, b);
        ratio[t] = r;
        if (r > bv) {  // NaN never wins
            bv = r;
            bi = t;
        }
    }
    // lexicographic (value desc, index asc) reduction
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(kFull, bv, o);
        const int oi = __shfl_down_sync(kFull, bi, o);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) {
            bv = ov;
            bi = oi;
        }
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane_id() == 0) {
        sv[w] = bv;
        si[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = -FLT_MAX;
        int i = -1;
        for (int k = 0; k < nw; ++k)
            if (si[k] >= 0 && (i < 0 || sv[k] > v || (sv[k] == v && si[k] < i))) {
                v = sv[k];
                i = si[k];
            }
        *best = i;
    }
}

// Per-cell update counts of one batch of measured beams: counts[2c] = hits that end in cell c
// (delta_occ), counts[2c+1] = beams that crossed c before their end (delta_emp). A beam whose
// range is at least max_range (or not finite) returned nothing: every cell up to max_range is
// crossed. The traversal is the evaluation's, cut at the measured range, so "the cell where the
// range ends" is decided by the same exact integer comparison as the range limit.
__global__ void __launch_bounds__(kWarpsExplore * 32)
    k_update_counts(int W, int H, const int32_t *__restrict__ poses, int P, const int32_t *__restrict__ dirs, int B,
                    const float *__restrict__ ranges, long long rfix_max, int cap, int stride,
                    uint32_t *__restrict__ counts, int *status)
{
    extern __shared__ float smem[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    float *sl = smem + (size_t)warp * 2 * stride;
    int *ids = (int *)(sl + stride);
    const long long nbeams = (long long)P * B;
    const unsigned ncell = (unsigned)W * (unsigned)H;
    for (long long beam = (long long)blockIdx.x * kWarpsExplore + warp; beam < nbeams;
         beam += (long long)gridDim.x * kWarpsExplore) {
        const int pi = (int)(beam / B), bi = (int)(beam % B);
        const float z = ranges[beam];
        if (!(z > 0.0f)) continue;  // no measurement (NaN or non-positive): no update
        // a return at z < max_range (decided on z's Q16 rounding, like the range limit itself)
        bool hit = false;
        long long rfix = rfix_max;
        if ((double)z < (double)rfix_max * (1.0 / 65536.0)) {
            const long long rz = __double2ll_rn((double)z * 65536.0);
            if (rz < rfix_max) {
                rfix = rz;
                hit = true;
            }
        }
        const int32_t *pose = poses + 4 * (size_t)pi;
        int dx, dy;
        beam_dir(pose, dirs[2 * bi], dirs[2 * bi + 1], dx, dy);
        const float rend = (float)((double)rfix * (1.0 / 65536.0));
        bool by_range = false;
        const int n = dda_warp(W, H, pose[0], pose[1], dx, dy, rfix, rend, cap, ids, sl, &by_range);
        if (n < 0) {
            if (lane == 0) set_status(status, FSMI_STATUS_BEAM_OVERFLOW);
            continue;
        }
        // a range that ends outside the grid hits no map cell: the crossed cells are still empty
        const bool inside = hit && by_range;
        for (int i = lane; i < n; i += 32) {
            const unsigned id = (unsigned)ids[i];
            if (id >= ncell) continue;
            const bool occ = inside && i == n - 1;
            atomicAdd(counts + 2 * (size_t)id + (occ ? 0 : 1), 1u);
        }
        __syncwarp();
    }
}

// o' = sigmoid(logit(o) + a ln delta_occ + b ln delta_emp) for cells with updates; o in {0, 1}
// stays put (infinite odds do not move).
__global__ void k_update_apply(float *__restrict__ map, long long ncell, const uint32_t *__restrict__ counts,
                               float log_docc, float log_demp)
{
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const uint2 k = reinterpret_cast<const uint2 *>(counts)[c];
        if ((k.x | k.y) == 0u) continue;
        const float o = map[c];
        if (!(o > 0.0f && o < 1.0f)) continue;
        const float lg = logf(o) - log1pf(-o) + (float)k.x * log_docc + (float)k.y * log_demp;
        map[c] = 1.0f / (1.0f + expf(-lg));
    }
}

int explore_grid(long long items, int per_block)
{
    long long g = (items + per_block - 1) / per_block;
    const long long gmax = (long long)sm_count() * 16;
    if (g > gmax) g = gmax;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_traj_stamps(int W, int H, const int32_t *poses, int P, const int32_t *traj_off, int T,
                               const int32_t *dirs, int B, long long rfix, float rend, int cap, int32_t *stamp,
                               int *status, cudaStream_t s)
{
    // every stamp starts above any state index (0x7f7f7f7f)
    cudaError_t e = cudaMemsetAsync(stamp, 0x7f, (size_t)T * W * H * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const long long nbeams = (long long)P * B;
    if (nbeams == 0) return cudaSuccess;
    const int stride = ((cap + 2) + 3) & ~3;
    const size_t smem = (size_t)kWarpsExplore * 2 * stride * sizeof(float);
    e = cudaFuncSetAttribute(k_traj_stamps, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_traj_stamps<<<explore_grid(nbeams, kWarpsExplore), kWarpsExplore * 32, smem, s>>>(
        W, H, poses, P, traj_off, T, dirs, B, rfix, rend, cap, stride, stamp, status);
    return cudaGetLastError();
}

cudaError_t launch_row_sums(const float *v, long long rows, int cols, float *out, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    k_row_sums<<<explore_grid(rows, 8), 256, 0, s>>>(v, rows, cols, out);
    return cudaGetLastError();
}

cudaError_t launch_csr_sums(const float *v, int nv, const int32_t *off, int nseg, float *out, cudaStream_t s)
{
    if (nseg <= 0) return cudaSuccess;
    k_csr_sums<<<explore_grid(nseg, 8), 256, 0, s>>>(v, nv, off, nseg, out);
    return cudaGetLastError();
}

cudaError_t launch_best_trajectory(const float *traj_mi, const int32_t *poses, int P, const int32_t *traj_off, int T,
                                   float *ratio, int32_t *best, cudaStream_t s)
{
    k_best_trajectory<<<1, 1024, 0, s>>>(traj_mi, poses, P, traj_off, T, ratio, best);
    return cudaGetLastError();
}

cudaError_t launch_update_map_2d(float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                                 const float *ranges, long long rfix, int cap, float log_docc, float log_demp,
                                 uint32_t *counts, int *status, cudaStream_t s)
{
    const long long ncell = (long long)W * H;
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)ncell * 2 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const long long nbeams = (long long)P * B;
    if (nbeams == 0) return cudaSuccess;
    const int stride = ((cap + 2) + 3) & ~3;
    const size_t smem = (size_t)kWarpsExplore * 2 * stride * sizeof(float);
    e = cudaFuncSetAttribute(k_update_counts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_update_counts<<<explore_grid(nbeams, kWarpsExplore), kWarpsExplore * 32, smem, s>>>(
        W, H, poses, P, dirs, B, ranges, rfix, cap, stride, counts, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_update_apply<<<explore_grid(ncell, 256), 256, 0, s>>>(map, ncell, counts, log_docc, log_demp);
    return cudaGetLastError();
}

cudaError_t prepare_explore()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_traj_stamps);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_row_sums);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_csr_sums);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_best_trajectory);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_update_counts);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_update_apply);
    return e;
}

}  // namespace fsmi
