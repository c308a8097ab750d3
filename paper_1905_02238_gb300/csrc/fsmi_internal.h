// Internal interface between the C-ABI layer (fsmi_api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fsmi {

// Host-validated parameters plus the derived constants every kernel needs.
struct DevParams {
    int variant;        // FSMI_EXACT / FSMI_APPROX / FSMI_UNIFORM
    float sigma;        // cells
    float inv_s2;       // 1 / (sigma * sqrt(2)): erfc argument scale of the 2D Gaussian tails
    float docc, demp;   // inverse sensor model odds factors
    int trunc;          // Delta
    int H;              // uniform half-width
    float inv_2h1;      // 1 / (2H + 1)
    long long rfix;     // round(max_range * 2^16), 2D range limit in Q16
    float rend;         // rfix / 2^16 as float: the end distance of a beam cut by the range
    int nmax;           // per-beam capacity: cells (2D) or virtual cells (3D)
    int e0;             // e0_mode
    int run_cap;        // RLE split length
    int g_kernel;       // FSMI_G_PDF / FSMI_G_ERF
    int approx_reading; // Approx-FSMI-RLE reading
    int K;              // RLE kernel support radius (cells)
    int flags;          // FSMI_FLAG_* bits
};

constexpr int kWarps2D = 4;   // warps per block, 2D kernels
constexpr int kWarpsRLE = 4;  // warps per block, RLE kernels

// 2D (fsmi_2d.cu)
cudaError_t launch_eval_2d(const float *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs,
                           int B, const DevParams &p, float *out, float4 *gains, int *status, cudaStream_t s);
cudaError_t launch_eval_beams(const int32_t *off, const float *o, const float *l, const float *lend, int nbeams,
                              const DevParams &p, float *out, int *status, cudaStream_t s);
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
                            const DevParams &p, float *out, int *status, cudaStream_t s);
cudaError_t launch_eval_3d(const Vox3D &v, const DevParams &p, float *out, int32_t *nruns, int *status,
                           cudaStream_t s);

// scan tile size of the RLE offsets (elements per tile)
constexpr int kScanTile = 4096;

// tile totals held by the library-owned scratch of fsmi_rle_encode_3d_noalloc (16 KiB, up to
// kEncodeScratchTiles * kScanTile rays per call)
constexpr int kEncodeScratchTiles = 4096;
cudaError_t launch_rle_encode_3d_static(const Vox3D &v, const DevParams &p, int32_t *run_off, float *run_o,
                                        uint8_t *run_len, int run_capacity, int ntiles, int *status,
                                        cudaStream_t s);

int sm_count();

}  // namespace fsmi
