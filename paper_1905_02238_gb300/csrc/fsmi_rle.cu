// RLE / 3D kernels and their launchers; the per-ray device code is in evalrle.cuh.
#include <cmath>
#include <mutex>

#include "evalrle.cuh"

namespace fsmi {

// MODE: kRay3dThm5 for Theorem 5's sub-blocks, kRay3dOther for every other variant (the launcher
// picks by thm5_of(p)), so that each kernel holds only the paths it can take; WIDE for batches of
// more than 2^31 - 1 rays (a 64-bit ray index division, which costs the others registers).
template <int MODE, bool WIDE>
__global__ void __launch_bounds__(kMaxWarps * 32)
    k_eval_3d(Vox3D vx, DevParams p, const __grid_constant__ RleTable tbl, long long nrays, int warp_floats,
              float *__restrict__ out, int32_t *__restrict__ nruns, unsigned long long *queue, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RleBlock rb = rle_block(smem_raw, p, tbl, warp_floats);
    for_each_item(nrays, queue, chunk, [&](long long ray) { eval_ray_3d<MODE, WIDE>(vx, p, rb, ray, out, nruns); });
}

__global__ void __launch_bounds__(kMaxWarps * 32)
    k_eval_rle(const int32_t *__restrict__ off, const float *__restrict__ ro, const uint8_t *__restrict__ rl,
               DevParams p, const __grid_constant__ RleTable tbl, long long nrays, int stride, float *__restrict__ out,
               int *status, unsigned long long *queue, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RleBlock rb = rle_block(smem_raw, p, tbl, kArraysRLE * stride);
    for_each_item(nrays, queue, chunk,
                  [&](long long ray) { eval_ray_rle(off, ro, rl, p, rb, stride, ray, out, status); });
}

__global__ void __launch_bounds__(kWarpsRLE * 32)
    k_rle_count(Vox3D vx, DevParams p, long long nrays, int stride, int32_t *__restrict__ run_off)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    float *O = (float *)smem_raw + (size_t)warp * 2 * stride;
    int *S = (int *)(O + stride);
    if (blockIdx.x == 0 && threadIdx.x == 0) run_off[0] = 0;
    for (long long ray = (long long)blockIdx.x * kWarpsRLE + warp; ray < nrays; ray += (long long)gridDim.x * kWarpsRLE) {
        const int nr = sample_encode(vx, ray, p.nmax, p.run_cap, O, S);
        if (lane_id() == 0) run_off[ray + 1] = nr;
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kWarpsRLE * 32)
    k_rle_write(Vox3D vx, DevParams p, long long nrays, int stride, const int32_t *__restrict__ run_off,
                float *__restrict__ run_o, uint8_t *__restrict__ run_len, int capacity, int *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    float *O = (float *)smem_raw + (size_t)warp * 2 * stride;
    int *S = (int *)(O + stride);
    for (long long ray = (long long)blockIdx.x * kWarpsRLE + warp; ray < nrays; ray += (long long)gridDim.x * kWarpsRLE) {
        const int nr = sample_encode(vx, ray, p.nmax, p.run_cap, O, S);
        const long long b = run_off[ray];  // saturated at INT32_MAX by the scan, never negative
        bool over = false;
        for (int u = lane; u < nr; u += 32) {
            const long long idx = b + u;
            if (idx >= 0 && idx < capacity) {
                run_o[idx] = O[u];
                run_len[idx] = (uint8_t)(S[u + 1] - S[u]);
            } else {
                over = true;
            }
        }
        if (__any_sync(kFull, over) && lane == 0) set_status(status, FSMI_STATUS_RUN_OVERFLOW);
        __syncwarp();
    }
}

// Inclusive scan of a[0..n) in tiles of kScanTile (1024 threads x 4), tile totals to tot[].
__device__ __forceinline__ int block_incl_scan(int v, int *wsum)
{
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    int x = warp_incl_add_int(v);
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
        w = warp_incl_add_int(w);
        wsum[lane] = w;
    }
    __syncthreads();
    if (warp > 0) x += wsum[warp - 1];
    __syncthreads();
    return x;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(int32_t *a, long long n, int32_t *tot)
{
    __shared__ int wsum[32];
    const long long t0 = (long long)blockIdx.x * kScanTile + 4LL * threadIdx.x;
    int v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (t0 + k < n) ? a[t0 + k] : 0;
        s += v[k];
    }
    const int ex = block_incl_scan(s, wsum) - s;
    int run = ex;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        run += v[k];
        if (t0 + k < n) a[t0 + k] = run;
    }
    if (threadIdx.x == blockDim.x - 1) tot[blockIdx.x] = run;
}

// 64-bit inclusive scan across the block (tile totals of up to 1024 tiles of 4096 rays can pass
// 2^31 runs, so they are summed in 64 bits)
__device__ __forceinline__ long long block_incl_scan_ll(long long v, long long *wsum)
{
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += t;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    if (warp > 0) x += wsum[warp - 1];
    __syncthreads();
    return x;
}

// Exclusive scan of the tile totals in place (one block, loops over chunks of 1024 tiles), summed
// in 64 bits. The offsets are int32: a tile whose runs start at or beyond INT32_MAX gets the
// start INT32_MAX, and FSMI_STATUS_RUN_OVERFLOW is set (k_scan_add saturates the offsets inside a
// tile the same way), so that no offset wraps to a negative value.
__global__ void __launch_bounds__(1024) k_scan_totals(int32_t *tot, int ntiles, int *status)
{
    __shared__ long long wsum[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    bool over = false;
    for (int b = 0; b < ntiles; b += 1024) {
        const int i = b + threadIdx.x;
        const long long v = i < ntiles ? (long long)tot[i] : 0;
        const long long inc = block_incl_scan_ll(v, wsum);
        const long long c = carry;
        if (i < ntiles) {
            const long long ex = c + inc - v;
            over |= c + inc > 0x7fffffffLL;
            tot[i] = (int32_t)min(ex, 0x7fffffffLL);
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + inc;
        __syncthreads();
    }
    if (over) set_status(status, FSMI_STATUS_RUN_OVERFLOW);
}

// offsets = tile-local inclusive sums + the tile's start, saturated at INT32_MAX
__global__ void k_scan_add(int32_t *a, long long n, const int32_t *tot)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = (int32_t)min((long long)a[i] + (long long)tot[i / kScanTile], 0x7fffffffLL);
}

// ---- launchers ---------------------------------------------------------------------------------

static int rle_stride(int nmax, int K) { return ((nmax + 2 * K + 4) + 3) & ~3; }  // cells + 2K padding

// The noise-kernel tables of one launch (RleTable), from g(d) = (1/(sqrt(2 pi) sigma))
// exp(-d^2 / (2 sigma^2)) (Theorem 3's density), the cell mass Phi((d + 1/2)/sigma) -
// Phi((d - 1/2)/sigma), or 1[|d| <= H] / (2H + 1) (Theorem 6), zero beyond the strict band.
void fill_rle_table(const DevParams &p, RleTable &t)
{
    const TabSpec ts = table_spec(p);
    const int K = ts.K;
    double g[FSMI_MAX_KERNEL_RADIUS + 1];
    const double s2 = ts.sigma * 1.4142135623730951;
    for (int a = 0; a <= K; ++a) {
        double v;
        if (ts.kind == 2)
            v = (a <= ts.H) ? 1.0 / (2.0 * ts.H + 1.0) : 0.0;
        else if (ts.kind == 1)
            v = 0.5 * (std::erfc(-(a + 0.5) / s2) - std::erfc(-(a - 0.5) / s2));
        else
            v = std::exp(-(double)a * a / (2.0 * ts.sigma * ts.sigma)) / (2.5066282746310002 * ts.sigma);
        if (ts.band >= 0 && a > ts.band) v = 0.0;
        g[a] = v;
        t.gtab[K + a] = (float)v;
        t.gtab[K - a] = (float)v;
    }
    double c0 = 0.0, c1 = 0.0;
    t.tab[0] = make_float2(0.0f, 0.0f);
    for (int d = -K; d <= K; ++d) {
        const double v = g[d < 0 ? -d : d];
        c0 += v;
        c1 += (double)d * v;
        t.tab[d + K + 1] = make_float2((float)c0, (float)(d == K ? 0.0 : c1));
    }
}

template <typename Kern>
static cudaError_t grid_for(Kern k, size_t smem, long long nitems, int wpb, int bps, long long &grid)
{
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (bps > 0 && bps < occ) occ = bps;
    const long long want = (nitems + wpb - 1) / wpb;
    grid = (long long)sm_count() * occ;
    if (grid > want) grid = want;
    if (grid < 1) grid = 1;
    return cudaSuccess;
}

static cudaError_t reset_queue(unsigned long long *queue, cudaStream_t s)
{
    return queue ? cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s) : cudaSuccess;
}

cudaError_t launch_eval_3d(const Vox3D &v, const DevParams &p, float *out, int32_t *nruns,
                           unsigned long long *queue, int *status, cudaStream_t s)
{
    (void)status;
    const long long nrays = (long long)v.P * v.R;
    if (nrays <= 0) return cudaSuccess;
    const Schedule &sc = current_schedule(FSMI_KIND_RLE);
    const int wf = ray3d_warp_floats(p);
    const size_t per_warp = (size_t)wf * sizeof(float);
    const int wpb = fit_warps(sc.warps_per_block, per_warp, rle_table_bytes(p.K));
    const size_t smem = rle_table_bytes(p.K) + (size_t)wpb * per_warp;
    long long grid;
    const bool wide = nrays > 0x7fffffffLL;
    auto kern = thm5_of(p) ? (wide ? k_eval_3d<kRay3dThm5, true> : k_eval_3d<kRay3dThm5, false>)
                           : (wide ? k_eval_3d<kRay3dOther, true> : k_eval_3d<kRay3dOther, false>);
    cudaError_t e = grid_for(kern, smem, nrays, wpb, sc.blocks_per_sm, grid);
    if (e == cudaSuccess) e = reset_queue(queue, s);
    if (e != cudaSuccess) return e;
    RleTable tbl;
    fill_rle_table(p, tbl);
    kern<<<(unsigned)grid, wpb * 32, smem, s>>>(v, p, tbl, nrays, wf, out, nruns, queue,
                                                sc.queue_chunk > 0 ? sc.queue_chunk : 1);
    return cudaGetLastError();
}

cudaError_t launch_eval_rle(const int32_t *run_off, const float *run_o, const uint8_t *run_len, int nrays,
                            const DevParams &p, float *out, unsigned long long *queue, int *status, cudaStream_t s)
{
    if (nrays <= 0) return cudaSuccess;
    const Schedule &sc = current_schedule(FSMI_KIND_RLE);
    const int stride = rle_stride(p.nmax, p.K);
    const size_t per_warp = (size_t)kArraysRLE * stride * sizeof(float);
    const int wpb = fit_warps(sc.warps_per_block, per_warp, rle_table_bytes(p.K));
    const size_t smem = rle_table_bytes(p.K) + (size_t)wpb * per_warp;
    long long grid;
    cudaError_t e = grid_for(k_eval_rle, smem, nrays, wpb, sc.blocks_per_sm, grid);
    if (e == cudaSuccess) e = reset_queue(queue, s);
    if (e != cudaSuccess) return e;
    RleTable tbl;
    fill_rle_table(p, tbl);
    k_eval_rle<<<(unsigned)grid, wpb * 32, smem, s>>>(run_off, run_o, run_len, p, tbl, nrays, stride, out, status,
                                                      queue, sc.queue_chunk > 0 ? sc.queue_chunk : 1);
    return cudaGetLastError();
}

cudaError_t launch_rle_encode_3d(const Vox3D &v, const DevParams &p, int32_t *run_off, float *run_o,
                                 uint8_t *run_len, int run_capacity, int32_t *ws_tiles, int ntiles, int *status,
                                 cudaStream_t s)
{
    const long long nrays = (long long)v.P * v.R;
    if (nrays <= 0) {
        return cudaMemsetAsync(run_off, 0, sizeof(int32_t), s);
    }
    const int stride = rle_stride(p.nmax, 0);
    const size_t smem = (size_t)kWarpsRLE * 2 * stride * sizeof(float);
    long long grid;
    cudaError_t e = grid_for(k_rle_count, smem, nrays, kWarpsRLE, 0, grid);
    if (e != cudaSuccess) return e;
    k_rle_count<<<(unsigned)grid, kWarpsRLE * 32, smem, s>>>(v, p, nrays, stride, run_off);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_scan_tiles<<<ntiles, 1024, 0, s>>>(run_off + 1, nrays, ws_tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_scan_totals<<<1, 1024, 0, s>>>(ws_tiles, ntiles, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    long long ag = (nrays + 255) / 256;
    if (ag > (long long)sm_count() * 8) ag = (long long)sm_count() * 8;
    k_scan_add<<<(unsigned)ag, 256, 0, s>>>(run_off + 1, nrays, ws_tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = grid_for(k_rle_write, smem, nrays, kWarpsRLE, 0, grid);
    if (e != cudaSuccess) return e;
    k_rle_write<<<(unsigned)grid, kWarpsRLE * 32, smem, s>>>(v, p, nrays, stride, run_off, run_o, run_len,
                                                              run_capacity, status);
    return cudaGetLastError();
}

// ---- run-length encoding without caller workspace -----------------------------------------
//
// Some callers cannot allocate device memory at the point where they encode rays: a planner that
// runs inside a real-time control loop with its device memory reserved up front, or host code
// that receives only input and output pointers from another framework and holds no allocator. For
// them the offset scan keeps its tile totals in this file-scope array instead of a caller
// workspace. Every GPU that loads the library holds it until the process exits.
__device__ __align__(256) int32_t g_encode_scan_scratch[kEncodeScratchTiles];

namespace {
std::mutex g_scratch_mu;
int32_t *g_scratch_ptr[64];
}  // namespace

cudaError_t encode_scratch_ptr(int32_t **ptr);

// Loads every RLE kernel on the current device (a kernel's first use loads it lazily).
cudaError_t prepare_rle()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_eval_3d<kRay3dThm5, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_3d<kRay3dOther, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_3d<kRay3dThm5, true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_3d<kRay3dOther, true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_rle);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_rle_count);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_rle_write);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_scan_tiles);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_scan_totals);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_scan_add);
    int32_t *scratch = nullptr;
    if (e == cudaSuccess) e = encode_scratch_ptr(&scratch);
    return e;
}

// Device address of g_encode_scan_scratch for the current device. The symbol's name is only a
// host-side stand-in, so the address is looked up once per device, with that device current.
cudaError_t encode_scratch_ptr(int32_t **ptr)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *a = nullptr;
        e = cudaGetSymbolAddress(&a, g_encode_scan_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = (int32_t *)a;
    }
    *ptr = g_scratch_ptr[dev];
    return cudaSuccess;
}

cudaError_t launch_rle_encode_3d_static(const Vox3D &v, const DevParams &p, int32_t *run_off, float *run_o,
                                        uint8_t *run_len, int run_capacity, int ntiles, int *status,
                                        cudaStream_t s)
{
    if (ntiles > kEncodeScratchTiles) return cudaErrorInvalidValue;
    int32_t *scratch = nullptr;
    cudaError_t e = encode_scratch_ptr(&scratch);
    if (e != cudaSuccess) return e;
    // the scan writes every tile total it reads, so the array needs no clearing between calls
    return launch_rle_encode_3d(v, p, run_off, run_o, run_len, run_capacity, scratch, ntiles, status, s);
}

}  // namespace fsmi
