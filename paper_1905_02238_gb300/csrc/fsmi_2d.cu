// 2D kernels and their launchers; the per-beam device code is in eval2d.cuh.
#include "eval2d.cuh"

namespace fsmi {

// Persistent kernel: each warp evaluates beams one at a time, either in a static grid-stride
// order or, with a work queue, taking `chunk` consecutive beams per atomic grab (balances beams
// of very different lengths). The queue counter must be zero at launch.
// Every variant fits in 64 registers (8 resident blocks of 4 warps, the shared-memory limit as
// well); the full sweep is the exact window loop with an unbounded window.
template <int VAR, int SRC>
__global__ void __launch_bounds__(kMaxWarps * 32, FSMI_MIN_BLOCKS_2D)
    k_eval_2d(Src2D src, DevParams p, long long nbeams, int stride, float *__restrict__ out, int *status,
              unsigned long long *queue, int chunk)
{
    extern __shared__ float smem[];
    const int lane = lane_id(), warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float *sl, *sc, *sp, *sx;
    carve_2d(smem + (size_t)warp * warp_floats_2d(stride), stride, sl, sc, sp, sx);
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
    const int stride = stride_2d(p.nmax);
    const size_t per_warp = (size_t)warp_floats_2d(stride) * sizeof(float);
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

cudaError_t map_gains(const float *map, int W, int H, const DevParams &p, float4 *gains, cudaStream_t s)
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
