// C ABI of libfsmi (include/fsmi.h): argument checks on the host, derived constants, the
// per-device status word, and dispatch to the kernel launchers.
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>

#include "../../include/fsmi.h"
#include "fsmi_internal.h"

namespace fsmi {

// Per-device status word (FSMI_STATUS_* bits), set by kernels with atomicOr.
__device__ int g_status;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int *g_status_ptr[kMaxDevices];
int g_sms[kMaxDevices];
int g_smem_optin[kMaxDevices];
thread_local int g_last_cuda = 0;

// defaults per family, from timing the schedule candidates on the 2D office-map batch and the
// 3D depth-camera batch: the queue removes the tail of the static assignment (the slowest of
// thousands of warps, each with its own mix of beam lengths)
constexpr Schedule kDefaults[2] = {{4, 0, 1, 32}, {2, 0, 4, 32}};
thread_local Schedule g_schedule[2] = {kDefaults[0], kDefaults[1]};

bool kind_ok(int kind) { return kind == FSMI_KIND_2D || kind == FSMI_KIND_RLE; }

int current_device()
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    return dev;
}

// Device address of g_status for the current device (looked up once per device with that
// device current; host code must not use the symbol itself as an address).
int *status_ptr()
{
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status) == cudaSuccess) g_status_ptr[dev] = (int *)p;
    }
    return g_status_ptr[dev];
}

fsmi_status cuda_fail(cudaError_t e)
{
    g_last_cuda = (int)e;
    return FSMI_ERR_CUDA;
}

bool finite_pos(float v) { return isfinite(v) && v > 0.0f; }

// Support radius of the RLE noise kernel: beyond 7.45 sigma the Gaussian is below 1e-12 of its
// peak, so the dropped terms change no FP32 result.
int gauss_radius(float sigma) { return (int)ceilf(7.45f * sigma); }

enum Use { kUse2D, kUseBeams, kUseRLE };

// ---- the per-cell gain as a Chebyshev series (RLE kernels) --------------------------------------

static double gain_exact(double d, double o)
{
    const double a = o * (d - 1.0), ria = 1.0 / (1.0 + a), omo = 1.0 - o, post = o * d * ria;
    return post * log1p((d - 1.0) * omo * ria) - omo * ria * log1p(a);
}

// gain_series of fsmi_device.cuh, operation for operation in FP32 (explicit fmaf, nothing left to
// contraction), so that the host sees exactly what the kernels compute
static float gain_series_host(const float *c, float o)
{
    const float x2 = fmaf(4.0f, o, -2.0f);
    float b1 = 0.0f, b2 = 0.0f;
    for (int k = kGainFitTerms - 1; k >= 1; --k) {
        const float t = c[k] - b2;
        const float b0 = fmaf(x2, b1, t);
        b2 = b1;
        b1 = b0;
    }
    const float hx = 0.5f * x2;
    const float t0 = c[0] - b2;
    const float h = fmaf(hx, b1, t0);
    const float om = 1.0f - o;
    const float w = o * om;
    return w * h;
}

// Fits h(o) = f(delta, o) / (o (1 - o)) for both deltas at Chebyshev nodes and keeps the series
// only if, evaluated as the kernels do, it is within 1e-6 of f (relative) everywhere on a dense
// grid of [0, 1] that includes points down to 1e-7 from either end; otherwise the kernels use the
// closed form. The last fit is remembered per host thread.
static void fit_gains(DevParams &d)
{
    thread_local float last_docc = -1.0f, last_demp = -1.0f, last_c[2][kGainFitTerms];
    thread_local int last_ok = 0;
    if (d.docc == last_docc && d.demp == last_demp) {
        d.gain_fit = last_ok;
        memcpy(d.gfit, last_c, sizeof(last_c));
        for (int k = 0; k < kGainFitTerms; ++k) {
            d.gfit2[k][0] = d.gfit[0][k];
            d.gfit2[k][1] = d.gfit[1][k];
        }
        return;
    }
    const int N = kGainFitTerms;
    const double pi = 3.14159265358979323846;
    bool ok = true;
    for (int w = 0; w < 2; ++w) {
        const double delta = w ? d.demp : d.docc;
        double h[kGainFitTerms];
        for (int j = 0; j < N; ++j) {
            const double oj = 0.5 * (cos(pi * (j + 0.5) / N) + 1.0);
            h[j] = gain_exact(delta, oj) / (oj * (1.0 - oj));
        }
        for (int k = 0; k < N; ++k) {
            double c = 0.0;
            for (int j = 0; j < N; ++j) c += h[j] * cos(pi * k * (j + 0.5) / N);
            d.gfit[w][k] = (float)(c * (k == 0 ? 1.0 : 2.0) / N);
        }
        auto check = [&](float o) {
            const double e = gain_exact(delta, (double)o);
            const double g = (double)gain_series_host(d.gfit[w], o);
            return e == 0.0 ? g == 0.0 : fabs(g - e) <= 1e-6 * fabs(e);
        };
        for (int i = 0; i <= 8192 && ok; ++i) ok = check((float)i / 8192.0f);
        for (double t = 1e-7; t < 1e-2 && ok; t *= 1.25) ok = check((float)t) && check((float)(1.0 - t));
    }
    d.gain_fit = ok ? 1 : 0;
    for (int k = 0; k < N; ++k) {
        d.gfit2[k][0] = d.gfit[0][k];
        d.gfit2[k][1] = d.gfit[1][k];
    }
    last_docc = d.docc;
    last_demp = d.demp;
    last_ok = d.gain_fit;
    memcpy(last_c, d.gfit, sizeof(last_c));
}

fsmi_status make_params(const fsmi_params *prm, Use use, DevParams &d)
{
    if (!prm) return FSMI_ERR_ARG;
    if (prm->variant < FSMI_EXACT || prm->variant > FSMI_UNIFORM) return FSMI_ERR_ARG;
    if (!finite_pos(prm->delta_occ) || !finite_pos(prm->delta_emp)) return FSMI_ERR_ARG;
    if (prm->variant != FSMI_UNIFORM && !finite_pos(prm->sigma)) return FSMI_ERR_ARG;
    if (prm->variant == FSMI_APPROX && prm->trunc_delta < 0) return FSMI_ERR_ARG;
    if (prm->variant == FSMI_UNIFORM && prm->uniform_h < 0) return FSMI_ERR_ARG;
    if (prm->e0_mode != 0 && prm->e0_mode != 1) return FSMI_ERR_ARG;
    if (prm->g_kernel != FSMI_G_PDF && prm->g_kernel != FSMI_G_ERF) return FSMI_ERR_ARG;
    if (prm->approx_reading != 0 && prm->approx_reading != 1) return FSMI_ERR_ARG;
    if (use != kUseBeams && !finite_pos(prm->max_range)) return FSMI_ERR_ARG;
    if (prm->flags & ~(FSMI_FLAG_FULL_SWEEP | FSMI_FLAG_FULL_WINDOW)) return FSMI_ERR_ARG;
    d.variant = prm->variant;
    d.sigma = prm->variant == FSMI_UNIFORM ? 1.0f : prm->sigma;
    d.inv_s2 = (float)(1.0 / ((double)d.sigma * 1.4142135623730951));
    d.docc = prm->delta_occ;
    d.demp = prm->delta_emp;
    d.trunc = prm->trunc_delta;
    d.H = prm->uniform_h;
    d.inv_2h1 = (float)(1.0 / (2.0 * prm->uniform_h + 1.0));
    d.e0 = prm->e0_mode;
    d.run_cap = prm->run_cap;
    d.g_kernel = prm->g_kernel;
    d.approx_reading = prm->approx_reading;
    d.flags = prm->flags;
    d.cell_runlen = g_schedule[FSMI_KIND_RLE].cell_runlen;
    d.rmax = prm->max_range;
    d.rfix = 0;
    d.rend = 0.0f;
    d.K = 0;
    d.gain_fit = 0;
    memset(d.gfit, 0, sizeof(d.gfit));
    memset(d.gfit2, 0, sizeof(d.gfit2));
    if (use == kUse2D) {
        if (prm->max_range > FSMI_MAX_RANGE_2D) return FSMI_ERR_CAPACITY;
        d.rfix = llrint((double)prm->max_range * 65536.0);
        d.rend = (float)((double)d.rfix / 65536.0);
        // a segment of length R crosses at most R(|cos| + |sin|) + 2 <= R sqrt(2) + 2 cells
        d.nmax = (int)((double)prm->max_range * 1.41421357) + 3;
    } else if (use == kUseBeams) {
        d.nmax = FSMI_MAX_CELLS;
    } else {
        const double ns = floor((double)prm->max_range);
        if (ns < 1.0) return FSMI_ERR_ARG;
        if (ns > FSMI_MAX_SAMPLES_3D) return FSMI_ERR_CAPACITY;
        d.nmax = (int)ns;
        if (prm->run_cap < 1 || prm->run_cap > 255) return FSMI_ERR_ARG;
        if (prm->variant == FSMI_UNIFORM) {
            d.K = prm->uniform_h;
        } else {
            d.K = gauss_radius(prm->sigma);
            if (d.K < 1) d.K = 1;
            if (prm->variant == FSMI_APPROX && prm->approx_reading == 1 && prm->trunc_delta < d.K) d.K = prm->trunc_delta;
        }
        if (d.K > FSMI_MAX_KERNEL_RADIUS) return FSMI_ERR_CAPACITY;
        fit_gains(d);
    }
    return FSMI_OK;
}

bool grid_ok(int v) { return v >= 1 && v <= FSMI_MAX_GRID; }

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// Work-queue counter at the front of a workspace, when the schedule asks for a queue and the
// workspace holds one.
unsigned long long *queue_of(int kind, void *ws, size_t ws_bytes)
{
    if (g_schedule[kind].queue_chunk <= 0 || !ws || !aligned16(ws) || ws_bytes < kQueueBytes) return nullptr;
    return (unsigned long long *)ws;
}

// Per-map-cell gains behind the queue counter, when the workspace fits them and the batch visits
// more cells (up to nbeams * nmax, half that on average) than the map holds.
float4 *gains_of(void *ws, size_t ws_bytes, long long cells, long long nbeams, int nmax)
{
    if (!ws || !aligned16(ws) || ws_bytes < kQueueBytes + (size_t)cells * sizeof(float4)) return nullptr;
    if (nbeams * (nmax / 2) < cells) return nullptr;
    return (float4 *)((char *)ws + kQueueBytes);
}

bool schedule_ok(const fsmi_schedule &s)
{
    return s.warps_per_block >= 0 && s.warps_per_block <= kMaxWarps && s.blocks_per_sm >= 0 && s.blocks_per_sm <= 64 &&
           s.queue_chunk >= -1 && s.queue_chunk <= 1 << 20 && s.cell_runlen >= 0 && s.cell_runlen <= 1 << 20;
}

Schedule to_internal(int kind, const fsmi_schedule &s)
{
    const Schedule &d = kDefaults[kind];
    Schedule r;
    r.warps_per_block = s.warps_per_block ? s.warps_per_block : d.warps_per_block;
    r.blocks_per_sm = s.blocks_per_sm;
    r.queue_chunk = s.queue_chunk ? s.queue_chunk : d.queue_chunk;
    r.cell_runlen = s.cell_runlen ? s.cell_runlen : d.cell_runlen;
    return r;
}

fsmi_schedule to_public(const Schedule &s)
{
    fsmi_schedule r;
    r.warps_per_block = s.warps_per_block;
    r.blocks_per_sm = s.blocks_per_sm;
    r.queue_chunk = s.queue_chunk;
    r.cell_runlen = s.cell_runlen;
    return r;
}
}  // namespace

fsmi_status record_cuda_error(cudaError_t e) { return cuda_fail(e); }

const Schedule &current_schedule(int kind) { return g_schedule[kind]; }

int sm_count()
{
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = v > 0 ? v : 1;
    }
    return g_sms[dev];
}

int fit_warps(int warps, size_t per_warp, size_t fixed)
{
    const int dev = current_device();
    int cap = 0;
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_smem_optin[dev]) {
            int v = 0;
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            g_smem_optin[dev] = v > 0 ? v : 48 * 1024;
        }
        cap = g_smem_optin[dev];
    }
    while (warps > 1 && fixed + (size_t)warps * per_warp > (size_t)cap) --warps;
    return warps;
}

}  // namespace fsmi

using namespace fsmi;

extern "C" {

fsmi_status fsmi_eval_2d(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                         const fsmi_params *prm, float *out, void *ws, size_t ws_bytes, fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUse2D, d);
    if (st != FSMI_OK) return st;
    if (!grid_ok(W) || !grid_ok(H) || P < 0 || B < 0) return FSMI_ERR_ARG;
    if ((long long)P * B == 0) return FSMI_OK;
    if (!map || !poses || !dirs || !out) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    const long long nbeams = (long long)P * B;
    cudaError_t e = launch_eval_2d(map, W, H, poses, P, dirs, B, d, out,
                                   gains_of(ws, ws_bytes, (long long)W * H, nbeams, d.nmax), queue_of(FSMI_KIND_2D, ws, ws_bytes), sp,
                                   (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_eval_2d_sets(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                              const fsmi_set_2d *sets, int nsets, long long nbeams, const fsmi_params *prm, float *out,
                              void *ws, size_t ws_bytes, fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUse2D, d);
    if (st != FSMI_OK) return st;
    if (!grid_ok(W) || !grid_ok(H) || P < 0 || B < 0 || nsets < 0 || nbeams < 0) return FSMI_ERR_ARG;
    if (nbeams == 0) return FSMI_OK;
    if (nsets == 0 || !map || !poses || !dirs || !sets || !out) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaError_t e = launch_eval_2d_sets(map, W, H, poses, P, dirs, B, sets, nsets, nbeams, d, out,
                                        gains_of(ws, ws_bytes, (long long)W * H, nbeams, d.nmax),
                                        queue_of(FSMI_KIND_2D, ws, ws_bytes), sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_trajectory_workspace_size(int W, int H, int T, size_t *bytes)
{
    if (!bytes || !grid_ok(W) || !grid_ok(H) || T < 0) return FSMI_ERR_ARG;
    const size_t cells = (size_t)W * H;
    *bytes = kQueueBytes + cells * sizeof(float4) + (size_t)T * cells * sizeof(int32_t);
    return FSMI_OK;
}

fsmi_status fsmi_eval_trajectories_2d(const float *map, int W, int H, const int32_t *poses, int P,
                                      const int32_t *traj_off, int T, const int32_t *dirs, int B, const fsmi_params *prm,
                                      float *beam_mi, float *state_mi, float *traj_mi, void *ws, size_t ws_bytes,
                                      fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUse2D, d);
    if (st != FSMI_OK) return st;
    if (!grid_ok(W) || !grid_ok(H) || P < 0 || B < 0 || T < 0) return FSMI_ERR_ARG;
    if (T == 0) return FSMI_OK;
    if (!map || !poses || !traj_off || !traj_mi || (P > 0 && (!state_mi || (B > 0 && (!dirs || !beam_mi)))))
        return FSMI_ERR_ARG;
    size_t need = 0;
    fsmi_trajectory_workspace_size(W, H, T, &need);
    if (!ws || !aligned16(ws) || ws_bytes < need) return FSMI_ERR_WORKSPACE;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaStream_t s = (cudaStream_t)stream;
    const long long cells = (long long)W * H;
    int32_t *stamp = (int32_t *)((char *)ws + kQueueBytes + (size_t)cells * sizeof(float4));
    cudaError_t e = launch_traj_stamps(W, H, poses, P, traj_off, T, dirs, B, d.rfix, d.rend, d.nmax, stamp, sp, s);
    if (e == cudaSuccess && (long long)P * B > 0)
        e = launch_eval_2d_traj(map, W, H, poses, P, traj_off, T, stamp, dirs, B, d, beam_mi,
                                gains_of(ws, ws_bytes, cells, (long long)P * B, d.nmax),
                                queue_of(FSMI_KIND_2D, ws, ws_bytes), sp, s);
    if (e == cudaSuccess && P > 0) {
        if (B > 0) e = launch_row_sums(beam_mi, P, B, state_mi, s);
        else e = cudaMemsetAsync(state_mi, 0, (size_t)P * sizeof(float), s);
    }
    if (e == cudaSuccess) e = launch_csr_sums(state_mi, P, traj_off, T, traj_mi, s);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_best_trajectory(const float *traj_mi, const int32_t *poses, int P, const int32_t *traj_off, int T,
                                 float *ratio, int32_t *best, fsmi_stream_t stream)
{
    if (T < 1 || P < 0 || !traj_mi || (P > 0 && !poses) || !traj_off || !ratio || !best) return FSMI_ERR_ARG;
    cudaError_t e = launch_best_trajectory(traj_mi, poses, P, traj_off, T, ratio, best, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_scan_sums(const float *beam_mi, long long P, int B, float *pose_mi, fsmi_stream_t stream)
{
    if (P < 0 || B < 0) return FSMI_ERR_ARG;
    if (P == 0) return FSMI_OK;
    if (!pose_mi || (B > 0 && !beam_mi)) return FSMI_ERR_ARG;
    cudaError_t e = B > 0 ? launch_row_sums(beam_mi, P, B, pose_mi, (cudaStream_t)stream)
                          : cudaMemsetAsync(pose_mi, 0, (size_t)P * sizeof(float), (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_update_map_2d(float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                               const float *ranges, const fsmi_params *prm, void *ws, size_t ws_bytes,
                               fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUse2D, d);
    if (st != FSMI_OK) return st;
    if (!grid_ok(W) || !grid_ok(H) || P < 0 || B < 0) return FSMI_ERR_ARG;
    if ((long long)P * B == 0) return FSMI_OK;
    if (!map || !poses || !dirs || !ranges) return FSMI_ERR_ARG;
    const size_t need = (size_t)W * H * 2 * sizeof(uint32_t);
    if (!ws || !aligned16(ws) || ws_bytes < need) return FSMI_ERR_WORKSPACE;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaError_t e = launch_update_map_2d(map, W, H, poses, P, dirs, B, ranges, d.rfix, d.nmax,
                                         (float)log((double)prm->delta_occ), (float)log((double)prm->delta_emp),
                                         (uint32_t *)ws, sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

// samples kept by a profile cut at max_range: i with i + 1/2 < max_range (all 256 if max_range <= 0)
static int profile_keep(float max_range)
{
    if (!(max_range > 0.0f)) return 256;
    const double k = ceil((double)max_range - 0.5);
    return k < 0.0 ? 0 : (k > 256.0 ? 256 : (int)k);
}

fsmi_status fsmi_profiles_2d(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                             float max_range, const int32_t *beam_ids, long long N, uint16_t *out,
                             fsmi_stream_t stream)
{
    if (!grid_ok(W) || !grid_ok(H) || P < 0 || B < 0 || N < 0 || max_range != max_range) return FSMI_ERR_ARG;
    if (!beam_ids && N != (long long)P * B) return FSMI_ERR_ARG;
    if (N == 0) return FSMI_OK;
    if (!map || !poses || !dirs || !out || B == 0) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaError_t e = launch_profiles(map, W, H, poses, P, dirs, B, profile_keep(max_range), beam_ids, N, out, sp,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_surrogate_workspace_size(int mode, long long N, size_t *bytes)
{
    if (!bytes || N < 0 || (mode != 0 && mode != 1)) return FSMI_ERR_ARG;
    if (mode == 0) {
        if (N > 65536) return FSMI_ERR_CAPACITY;
        *bytes = surrogate_train_floats((int)N) * sizeof(float);
    } else {
        *bytes = surrogate_infer_bytes(N);
    }
    return FSMI_OK;
}

fsmi_status fsmi_surrogate_loss_grad(const float *params, const uint16_t *wbf16, const uint16_t *x, const float *y,
                                     int N, float *grad, float *loss, float *pred, void *ws, size_t ws_bytes,
                                     fsmi_stream_t stream)
{
    if (N < 1 || N > 65536 || !params || !wbf16 || !x) return FSMI_ERR_ARG;
    if (y && (!grad || !loss)) return FSMI_ERR_ARG;
    if (!y && !pred) return FSMI_ERR_ARG;
    if (!ws || !aligned16(ws) || ws_bytes < surrogate_train_floats(N) * sizeof(float)) return FSMI_ERR_WORKSPACE;
    cudaError_t e = launch_surrogate_loss_grad(params, wbf16, x, y, N, grad, loss, pred, (float *)ws,
                                               (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_surrogate_adam(float *params, float *m, float *v, const float *grad, float lr, float beta1,
                                float beta2, float eps, int t, uint16_t *wbf16, fsmi_stream_t stream)
{
    if (!params || !m || !v || !grad || !wbf16 || t < 1 || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
        return FSMI_ERR_ARG;
    cudaError_t e = launch_surrogate_adam(params, m, v, grad, lr, beta1, beta2, eps, t, wbf16, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_surrogate_cast(const float *params, uint16_t *wbf16, fsmi_stream_t stream)
{
    if (!params || !wbf16) return FSMI_ERR_ARG;
    cudaError_t e = launch_surrogate_cast(params, wbf16, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_surrogate_predict(const float *params, const uint16_t *wbf16, const float *map, int W, int H,
                                   const int32_t *poses, int P, const int32_t *dirs, int B, float max_range,
                                   const uint16_t *x, long long N, float *pred, void *ws, size_t ws_bytes,
                                   fsmi_stream_t stream)
{
    if (!params || !wbf16 || !pred || max_range != max_range) return FSMI_ERR_ARG;
    if (map) {
        if (!grid_ok(W) || !grid_ok(H) || P < 0 || B < 0 || (P > 0 && B > 0 && (!poses || !dirs))) return FSMI_ERR_ARG;
        N = (long long)P * B;
    } else if (N < 0 || (N > 0 && !x)) {
        return FSMI_ERR_ARG;
    }
    if (N == 0) return FSMI_OK;
    if (!ws || !aligned16(ws) || ws_bytes < surrogate_infer_bytes(N)) return FSMI_ERR_WORKSPACE;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaError_t e = launch_surrogate_infer(map, W, H, poses, dirs, B, profile_keep(max_range), x, N, wbf16, params,
                                           pred, ws, sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_topk(const float *v, int n, int k, int32_t *idx, fsmi_stream_t stream)
{
    if (!v || !idx || n < 1 || n > 16384 || k < 1 || k > n) return FSMI_ERR_ARG;
    cudaError_t e = launch_topk(v, n, k, idx, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_gather_rows(const int32_t *src, long long nrows, int width, const int32_t *idx, int k, int32_t *dst,
                             fsmi_stream_t stream)
{
    if (width < 1 || k < 0 || nrows < 0 || (k > 0 && (!src || !idx || !dst))) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaError_t e = launch_gather_rows(src, nrows, width, idx, k, dst, sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_eval_mixed(const float *map, int W, int H, const int32_t *poses2, int P2, const int32_t *dirs2, int B2,
                            const fsmi_params *prm2, const fsmi_volume *vols, int nvol, const int32_t *poses3, int P3,
                            const int32_t *dirs3, int R3, const fsmi_params *prm3, const fsmi_set *sets, int nsets,
                            long long nitems, float *out, unsigned long long *times, void *ws, size_t ws_bytes,
                            fsmi_stream_t stream)
{
    DevParams d2, d3;
    if (prm2) {
        fsmi_status st = make_params(prm2, kUse2D, d2);
        if (st != FSMI_OK) return st;
        if (!grid_ok(W) || !grid_ok(H) || P2 < 0 || B2 < 0 || !map || (P2 > 0 && !poses2) || (B2 > 0 && !dirs2))
            return FSMI_ERR_ARG;
    }
    if (prm3) {
        fsmi_status st = make_params(prm3, kUseRLE, d3);
        if (st != FSMI_OK) return st;
        if (nvol < 0 || P3 < 0 || R3 < 0 || (nvol > 0 && !vols) || (P3 > 0 && !poses3) || (R3 > 0 && !dirs3))
            return FSMI_ERR_ARG;
    }
    if (nsets < 0 || nitems < 0) return FSMI_ERR_ARG;
    if (nitems == 0) return FSMI_OK;
    if (nsets == 0 || !sets || !out || (!prm2 && !prm3)) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaStream_t s = (cudaStream_t)stream;
    float4 *gains = prm2 ? gains_of(ws, ws_bytes, (long long)W * H, nitems, d2.nmax) : nullptr;
    // the range-class plan, when the workspace holds it (fsmi_mixed_workspace_size)
    const size_t plan_at = kQueueBytes + (prm2 ? (size_t)W * H * sizeof(float4) : 0);
    unsigned char *plan = (ws && aligned16(ws) && ws_bytes >= plan_at + mixed_plan_bytes(nsets))
                              ? (unsigned char *)ws + plan_at
                              : nullptr;
    cudaError_t e = cudaSuccess;
    if (gains) e = map_gains(map, W, H, d2, gains, s);
    if (e == cudaSuccess)
        e = launch_eval_mixed(map, W, H, gains, poses2, P2, dirs2, B2, prm2 ? &d2 : nullptr, vols, nvol, poses3, P3,
                              dirs3, R3, prm3 ? &d3 : nullptr, sets, nsets, nitems, out, times, sp,
                              queue_of(FSMI_KIND_2D, ws, ws_bytes), plan, s);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_mixed_workspace_size(long long map_cells, int nsets, size_t *bytes)
{
    if (!bytes || map_cells < 0 || nsets < 0) return FSMI_ERR_ARG;
    *bytes = kQueueBytes + (size_t)map_cells * sizeof(float4) + mixed_plan_bytes(nsets);
    return FSMI_OK;
}

fsmi_status fsmi_eval_beams(const int32_t *off, const float *o, const float *l, const float *lend, int nbeams,
                            const fsmi_params *prm, float *out, void *ws, size_t ws_bytes, fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUseBeams, d);
    if (st != FSMI_OK) return st;
    if (nbeams < 0) return FSMI_ERR_ARG;
    if (nbeams == 0) return FSMI_OK;
    if (!off || !o || !l || !lend || !out) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaError_t e = launch_eval_beams(off, o, l, lend, nbeams, d, out, queue_of(FSMI_KIND_2D, ws, ws_bytes), sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_trace_2d(int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B, float max_range,
                          int cap, int32_t *cells, float *l, int32_t *n, fsmi_stream_t stream)
{
    if (!grid_ok(W) || !grid_ok(H) || P < 0 || B < 0 || cap < 1) return FSMI_ERR_ARG;
    if (!isfinite(max_range) || max_range <= 0.0f) return FSMI_ERR_ARG;
    if (max_range > FSMI_MAX_RANGE_2D) return FSMI_ERR_CAPACITY;
    if ((long long)P * B == 0) return FSMI_OK;
    if (!poses || !dirs || !cells || !l || !n) return FSMI_ERR_ARG;
    const long long rfix = llrint((double)max_range * 65536.0);
    cudaError_t e = launch_trace_2d(W, H, poses, P, dirs, B, rfix, (float)((double)rfix / 65536.0), cap, cells, l, n,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

static bool vox_ok(const float *vox, int X, int Y, int Z, const int32_t *poses, int P, const int32_t *dirs, int R)
{
    return grid_ok(X) && grid_ok(Y) && grid_ok(Z) && P >= 0 && R >= 0 &&
           ((long long)P * R == 0 || (vox && poses && dirs));
}

static long long scan_tiles(long long nitems) { return (nitems + kScanTile - 1) / kScanTile; }

fsmi_status fsmi_rle_encode_3d(const float *vox, int X, int Y, int Z, const int32_t *poses, int P,
                               const int32_t *dirs, int R, const fsmi_params *prm, int32_t *run_off, float *run_o,
                               uint8_t *run_len, int run_capacity, void *ws, size_t ws_bytes, fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUseRLE, d);
    if (st != FSMI_OK) return st;
    if (!vox_ok(vox, X, Y, Z, poses, P, dirs, R) || run_capacity < 0 || !run_off) return FSMI_ERR_ARG;
    const long long nrays = (long long)P * R;
    if (nrays > 0x7ffffffeLL) return FSMI_ERR_CAPACITY;
    if (run_capacity > 0 && (!run_o || !run_len)) return FSMI_ERR_ARG;
    const long long ntiles = scan_tiles(nrays);
    if (ntiles > 0 && (!ws || ws_bytes < (size_t)ntiles * sizeof(int32_t) || ((uintptr_t)ws & 3))) return FSMI_ERR_WORKSPACE;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    Vox3D v{vox, X, Y, Z, poses, P, dirs, R};
    cudaError_t e = launch_rle_encode_3d(v, d, run_off, run_o, run_len, run_capacity, (int32_t *)ws, (int)ntiles, sp,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_rle_encode_3d_noalloc(const float *vox, int X, int Y, int Z, const int32_t *poses, int P,
                                       const int32_t *dirs, int R, const fsmi_params *prm, int32_t *run_off,
                                       float *run_o, uint8_t *run_len, int run_capacity, fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUseRLE, d);
    if (st != FSMI_OK) return st;
    if (!vox_ok(vox, X, Y, Z, poses, P, dirs, R) || run_capacity < 0 || !run_off) return FSMI_ERR_ARG;
    const long long nrays = (long long)P * R;
    if (nrays > FSMI_NOALLOC_MAX_RAYS) return FSMI_ERR_CAPACITY;
    if (run_capacity > 0 && (!run_o || !run_len)) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    Vox3D v{vox, X, Y, Z, poses, P, dirs, R};
    cudaError_t e = launch_rle_encode_3d_static(v, d, run_off, run_o, run_len, run_capacity, (int)scan_tiles(nrays),
                                                sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_eval_rle(const int32_t *run_off, const float *run_o, const uint8_t *run_len, int nrays,
                          const fsmi_params *prm, float *out, void *ws, size_t ws_bytes, fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUseRLE, d);
    if (st != FSMI_OK) return st;
    if (nrays < 0) return FSMI_ERR_ARG;
    if (nrays == 0) return FSMI_OK;
    if (!run_off || !run_o || !run_len || !out) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    cudaError_t e =
        launch_eval_rle(run_off, run_o, run_len, nrays, d, out, queue_of(FSMI_KIND_RLE, ws, ws_bytes), sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_eval_3d(const float *vox, int X, int Y, int Z, const int32_t *poses, int P, const int32_t *dirs,
                         int R, const fsmi_params *prm, float *out, int32_t *nruns, void *ws, size_t ws_bytes,
                         fsmi_stream_t stream)
{
    DevParams d;
    fsmi_status st = make_params(prm, kUseRLE, d);
    if (st != FSMI_OK) return st;
    if (!vox_ok(vox, X, Y, Z, poses, P, dirs, R)) return FSMI_ERR_ARG;
    if ((long long)P * R == 0) return FSMI_OK;
    if (!out) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    Vox3D v{vox, X, Y, Z, poses, P, dirs, R};
    cudaError_t e = launch_eval_3d(v, d, out, nruns, queue_of(FSMI_KIND_RLE, ws, ws_bytes), sp, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_gauss_tail(const float *s, float *out, long long n, fsmi_stream_t stream)
{
    if (n < 0) return FSMI_ERR_ARG;
    if (n == 0) return FSMI_OK;
    if (!s || !out) return FSMI_ERR_ARG;
    cudaError_t e = launch_gauss_tail(s, out, n, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_workspace_size(int fn, long long nitems, const fsmi_params *prm, size_t *bytes)
{
    (void)prm;
    if (!bytes || nitems < 0) return FSMI_ERR_ARG;
    *bytes = 0;
    if (fn < FSMI_FN_EVAL_2D || fn > FSMI_FN_UPDATE_MAP_2D) return FSMI_ERR_ARG;
    if (fn == FSMI_FN_RLE_ENCODE_3D) *bytes = (size_t)scan_tiles(nitems) * sizeof(int32_t);
    else if (fn == FSMI_FN_EVAL_2D) *bytes = kQueueBytes + (size_t)nitems * sizeof(float4);
    else if (fn == FSMI_FN_UPDATE_MAP_2D) *bytes = (size_t)nitems * 2 * sizeof(uint32_t);
    else *bytes = kQueueBytes;
    return FSMI_OK;
}

fsmi_status fsmi_set_wait_limit(long long polls)
{
    set_epilogue_polls(polls);
    return FSMI_OK;
}

fsmi_status fsmi_device_status(fsmi_stream_t stream, int *status)
{
    if (!status) return FSMI_ERR_ARG;
    int *sp = status_ptr();
    if (!sp) return cuda_fail(cudaGetLastError());
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, sp, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sp, 0, sizeof(int), (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e);
    *status = v;
    return FSMI_OK;
}

const char *fsmi_status_str(fsmi_status s)
{
    switch (s) {
        case FSMI_OK: return "ok";
        case FSMI_ERR_ARG: return "invalid argument";
        case FSMI_ERR_CAPACITY: return "size exceeds a documented maximum";
        case FSMI_ERR_CUDA: return "CUDA error";
        case FSMI_ERR_TIMEOUT: return "device wait timed out";
        case FSMI_ERR_WORKSPACE: return "workspace too small";
        default: return "unknown status";
    }
}

fsmi_status fsmi_set_schedule(int kind, const fsmi_schedule *sched)
{
    if (!kind_ok(kind)) return FSMI_ERR_ARG;
    if (!sched) {
        g_schedule[kind] = kDefaults[kind];
        return FSMI_OK;
    }
    if (!schedule_ok(*sched)) return FSMI_ERR_ARG;
    g_schedule[kind] = to_internal(kind, *sched);
    return FSMI_OK;
}

fsmi_status fsmi_get_schedule(int kind, fsmi_schedule *sched)
{
    if (!kind_ok(kind) || !sched) return FSMI_ERR_ARG;
    *sched = to_public(g_schedule[kind]);
    return FSMI_OK;
}

fsmi_status fsmi_schedule_candidates(int kind, fsmi_schedule *out, int max, int *n)
{
    if (!kind_ok(kind) || max < 0 || !n || (max > 0 && !out)) return FSMI_ERR_ARG;
    static const int kWpb2D[] = {2, 4, 8}, kChunk2D[] = {1, 4, -1};
    static const int kWpbRLE[] = {1, 2, 4}, kChunkRLE[] = {2, 4, 8, -1}, kRunlen[] = {16, 32};
    int k = 0;
    auto put = [&](int w, int c, int r) {
        if (k < max) out[k] = to_public(to_internal(kind, fsmi_schedule{w, 0, c, r}));
        ++k;
    };
    if (kind == FSMI_KIND_2D) {
        for (int w : kWpb2D)
            for (int c : kChunk2D) put(w, c, 0);
    } else {
        for (int w : kWpbRLE)
            for (int c : kChunkRLE)
                for (int r : kRunlen) put(w, c, r);
    }
    *n = k < max ? k : max;
    return FSMI_OK;
}

fsmi_status fsmi_autotune(int kind, fsmi_tune_fn fn, void *ctx, const fsmi_schedule *cands, int ncands, int reps,
                          fsmi_stream_t stream, fsmi_schedule *best, float *ms)
{
    if (!kind_ok(kind) || !fn || !cands || ncands < 1 || reps < 1 || !best) return FSMI_ERR_ARG;
    for (int i = 0; i < ncands; ++i)
        if (!schedule_ok(cands[i])) return FSMI_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e);
    }
    const Schedule saved = g_schedule[kind];
    int ibest = -1;
    float tbest = 0.0f;
    for (int i = 0; i < ncands; ++i) {
        g_schedule[kind] = to_internal(kind, cands[i]);
        float t = -1.0f;
        bool ok = fn(ctx, stream) == FSMI_OK;
        ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
        for (int r = 0; ok && r < reps; ++r) ok = fn(ctx, stream) == FSMI_OK;
        ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
        t = ok ? t / reps : -1.0f;
        if (ms) ms[i] = t;
        if (ok && (ibest < 0 || t < tbest)) {
            ibest = i;
            tbest = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ibest < 0) {
        g_schedule[kind] = saved;
        return FSMI_ERR_ARG;
    }
    g_schedule[kind] = to_internal(kind, cands[ibest]);
    *best = to_public(g_schedule[kind]);
    return FSMI_OK;
}

fsmi_status fsmi_prepare(void)
{
    if (!status_ptr()) return cuda_fail(cudaGetLastError());
    (void)sm_count();
    (void)fit_warps(1, 0, 0);
    cudaError_t e = prepare_2d();
    if (e == cudaSuccess) e = prepare_rle();
    if (e == cudaSuccess) e = prepare_explore();
    if (e == cudaSuccess) e = prepare_surrogate();
    if (e == cudaSuccess) e = prepare_mixed();
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

struct fsmi_graph_st {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

fsmi_status fsmi_capture_begin(fsmi_stream_t stream)
{
    if (!stream) return FSMI_ERR_ARG;
    cudaError_t e = cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_capture_end(fsmi_stream_t stream, fsmi_graph *graph)
{
    if (!stream || !graph) return FSMI_ERR_ARG;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture((cudaStream_t)stream, &g);
    if (e != cudaSuccess) return cuda_fail(e);
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    fsmi_graph_st *h = new (std::nothrow) fsmi_graph_st{g, x};
    if (!h) {
        cudaGraphExecDestroy(x);
        cudaGraphDestroy(g);
        return FSMI_ERR_CAPACITY;
    }
    *graph = h;
    return FSMI_OK;
}

fsmi_status fsmi_graph_launch(fsmi_graph graph, fsmi_stream_t stream)
{
    if (!graph) return FSMI_ERR_ARG;
    cudaError_t e = cudaGraphLaunch(graph->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

fsmi_status fsmi_graph_destroy(fsmi_graph graph)
{
    if (!graph) return FSMI_ERR_ARG;
    cudaError_t e = cudaGraphExecDestroy(graph->exec);
    cudaError_t e2 = cudaGraphDestroy(graph->graph);
    delete graph;
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? FSMI_OK : cuda_fail(e);
}

int fsmi_last_cuda_error(void) { return g_last_cuda; }

int fsmi_version(void) { return 200; }

}  // extern "C"
