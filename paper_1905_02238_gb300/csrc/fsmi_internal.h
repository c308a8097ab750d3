// Internal interface between the C-ABI layer (fsmi_api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fsmi.h"

namespace fsmi {

// Host-validated parameters plus the derived constants every kernel needs.
constexpr int kGainFitTerms = 14;  // terms of the Chebyshev series of the per-cell gain (degree 13)

struct DevParams {
    int variant;        // FSMI_EXACT / FSMI_APPROX / FSMI_UNIFORM
    float sigma;        // cells
    float inv_s2;       // 1 / (sigma * sqrt(2)): erfc argument scale of the 2D Gaussian tails
    float docc, demp;   // inverse sensor model odds factors
    int trunc;          // Delta
    int H;              // uniform half-width
    float inv_2h1;      // 1 / (2H + 1)
    long long rfix;     // round(max_range * 2^16), 2D range limit in Q16
    float rmax;         // max_range as given (2D: bound of a candidate set's range)
    float rend;         // rfix / 2^16 as float: the end distance of a beam cut by the range
    int nmax;           // per-beam capacity: cells (2D) or virtual cells (3D)
    int e0;             // e0_mode
    int run_cap;        // RLE split length
    int g_kernel;       // FSMI_G_PDF / FSMI_G_ERF
    int approx_reading; // Approx-FSMI-RLE reading
    int K;              // RLE kernel support radius (cells)
    int flags;          // FSMI_FLAG_* bits
    int cell_runlen;    // RLE: rays whose mean run length is below this take the cell-level form
    // Chebyshev series of h(o) = f(delta, o) / (o (1 - o)) on [0, 1] for delta_occ ([0]) and
    // delta_emp ([1]), used by the RLE kernels when gain_fit is set (see gain_series)
    int gain_fit;
    float gfit[2][kGainFitTerms];
    float gfit2[kGainFitTerms][2];  // the same coefficients interleaved (delta_occ, delta_emp) per term
};

// Noise-kernel tables of the RLE kernels for radius K = table_spec(p).K (fill_rle_table, on the
// host in double, once per launch): tab[d + K + 1] = (sum_{e <= d} g(e), sum_{e <= d} e g(e))
// for d = -K-1..K (tab[0] = 0, the second sum 0 at d = K), gtab[K + d] = g(d), d = -K..K.
struct RleTable {
    float2 tab[2 * FSMI_MAX_KERNEL_RADIUS + 2];
    float gtab[2 * FSMI_MAX_KERNEL_RADIUS + 1];
};
void fill_rle_table(const DevParams &p, RleTable &t);

constexpr int kMaxWarps = 8;  // most warps per block any evaluation kernel is launched with
constexpr int kWarpsRLE = 4;  // warps per block of the RLE encoder kernels

// Launch schedule of one kernel family (fsmi_set_schedule; defaults filled in).
struct Schedule {
    int warps_per_block;  // 1 .. kMaxWarps
    int blocks_per_sm;    // 0 = as many as fit
    int queue_chunk;      // beams per queue grab; -1 = static assignment
    int cell_runlen;      // >= 1 (RLE family)
};
const Schedule &current_schedule(int kind);  // FSMI_KIND_2D / FSMI_KIND_RLE

// The schedule's warps per block, lowered until `fixed` + warps * `per_warp` bytes of shared
// memory fit in one block of the current device (at least 1).
int fit_warps(int warps, size_t per_warp, size_t fixed);

// Bytes at the front of an evaluation workspace reserved for the work-queue counter.
constexpr size_t kQueueBytes = 256;

// 2D (fsmi_2d.cu)
cudaError_t launch_eval_2d(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                           const DevParams &p, float *out, float4 *gains, unsigned long long *queue, int *status,
                           cudaStream_t s);
cudaError_t launch_eval_2d_sets(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs,
                                int B, const fsmi_set_2d *sets, int nsets, long long nbeams, const DevParams &p, float *out,
                                float4 *gains, unsigned long long *queue, int *status, cudaStream_t s);
cudaError_t launch_eval_2d_traj(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *traj_off,
                                int T, const int32_t *stamp, const int32_t *dirs, int B, const DevParams &p, float *out,
                                float4 *gains, unsigned long long *queue, int *status, cudaStream_t s);
cudaError_t map_gains(const float *map, int W, int H, const DevParams &p, float4 *gains, cudaStream_t s);
cudaError_t launch_eval_beams(const int32_t *off, const float *o, const float *l, const float *lend, int nbeams,
                              const DevParams &p, float *out, unsigned long long *queue, int *status, cudaStream_t s);
cudaError_t launch_trace_2d(int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B, long long rfix,
                            float rend, int cap, int32_t *cells, float *l, int32_t *n, cudaStream_t s);
cudaError_t launch_gauss_tail(const float *s, float *out, long long n, cudaStream_t st);

// 3D / RLE (fsmi_rle.cu)
struct Vox3D {
    const float *vox;
    int X, Y, Z;
    const int32_t *poses;
    int P;
    const int32_t *dirs;
    int R;
};
cudaError_t launch_rle_encode_3d(const Vox3D &v, const DevParams &p, int32_t *run_off, float *run_o,
                                 uint8_t *run_len, int run_capacity, int32_t *ws_tiles, int ntiles, int *status,
                                 cudaStream_t s);
cudaError_t launch_eval_rle(const int32_t *run_off, const float *run_o, const uint8_t *run_len, int nrays,
                            const DevParams &p, float *out, unsigned long long *queue, int *status, cudaStream_t s);
cudaError_t launch_eval_3d(const Vox3D &v, const DevParams &p, float *out, int32_t *nruns,
                           unsigned long long *queue, int *status, cudaStream_t s);

// scan tile size of the RLE offsets (elements per tile)
constexpr int kScanTile = 4096;

// tile totals held by the library-owned scratch of fsmi_rle_encode_3d_noalloc (16 KiB, up to
// kEncodeScratchTiles * kScanTile rays per call)
constexpr int kEncodeScratchTiles = 4096;
cudaError_t launch_rle_encode_3d_static(const Vox3D &v, const DevParams &p, int32_t *run_off, float *run_o,
                                        uint8_t *run_len, int run_capacity, int ntiles, int *status,
                                        cudaStream_t s);

int sm_count();
// records e as the calling thread's last CUDA error and returns FSMI_ERR_CUDA
fsmi_status record_cuda_error(cudaError_t e);
// poll limit of the surrogate fc kernel's epilogue wait for this host thread (< 0: the default)
void set_epilogue_polls(long long polls);

// exploration loop (fsmi_explore.cu): trajectory visit stamps and sums, the Bayesian map update
cudaError_t launch_traj_stamps(int W, int H, const int32_t *poses, int P, const int32_t *traj_off, int T,
                               const int32_t *dirs, int B, long long rfix, float rend, int cap, int32_t *stamp,
                               int *status, cudaStream_t s);
cudaError_t launch_row_sums(const float *v, long long rows, int cols, float *out, cudaStream_t s);
cudaError_t launch_csr_sums(const float *v, int nv, const int32_t *off, int nseg, float *out, cudaStream_t s);
cudaError_t launch_best_trajectory(const float *traj_mi, const int32_t *poses, int P, const int32_t *traj_off, int T,
                                   float *ratio, int32_t *best, cudaStream_t s);
cudaError_t launch_update_map_2d(float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                                 const float *ranges, long long rfix, int cap, float log_docc, float log_demp,
                                 uint32_t *counts, int *status, cudaStream_t s);
cudaError_t prepare_explore();

// mixed 2D / 3D candidate sets in one launch (fsmi_mixed.cu)
cudaError_t launch_eval_mixed(const float *map, int W, int H, const float4 *gains, const int32_t *poses2, int P2,
                              const int32_t *dirs2, int B2, const DevParams *p2, const fsmi_volume *vols, int nvol,
                              const int32_t *poses3, int P3, const int32_t *dirs3, int R3, const DevParams *p3,
                              const fsmi_set *sets, int nsets, long long nitems, float *out, unsigned long long *times,
                              int *status, unsigned long long *queue, unsigned char *plan, cudaStream_t s);
// bytes of the range-class plan of fsmi_eval_mixed for nsets sets (8-byte aligned start)
size_t mixed_plan_bytes(int nsets);
cudaError_t prepare_mixed();

// learned surrogate (fsmi_surrogate.cu)
size_t surrogate_train_floats(int N);
size_t surrogate_infer_bytes(long long N);
// profiles keep samples i < keep (the rest read as outside the map)
cudaError_t launch_profiles(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                            int keep, const int32_t *beam_ids, long long N, void *out, int *status, cudaStream_t s);
cudaError_t launch_surrogate_loss_grad(const float *params, const void *wbf16, const void *x, const float *y, int N,
                                       float *grad, float *loss, float *pred_out, float *ws, cudaStream_t s);
cudaError_t launch_surrogate_adam(float *p, float *m, float *v, const float *g, float lr, float b1, float b2, float eps,
                                  int t, void *wbf16, cudaStream_t s);
cudaError_t launch_surrogate_cast(const float *p, void *wbf16, cudaStream_t s);
cudaError_t launch_surrogate_infer(const float *map, int W, int H, const int32_t *poses, const int32_t *dirs, int B,
                                   int keep, const void *x, long long N, const void *wbf16, const float *params,
                                   float *pred, void *ws, int *status, cudaStream_t s);
cudaError_t launch_topk(const float *v, int n, int k, int32_t *idx, cudaStream_t s);
cudaError_t launch_gather_rows(const int32_t *src, long long nrows, int width, const int32_t *idx, int k,
                               int32_t *dst, int *status, cudaStream_t s);
cudaError_t prepare_surrogate();

// kernel loads and per-device lookups done ahead of stream capture (fsmi_prepare)
cudaError_t prepare_2d();
cudaError_t prepare_rle();

}  // namespace fsmi
