/*
 * fsmi.h - C ABI of libfsmi: batched Shannon mutual information between an occupancy map and
 * range beams, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Zhang, Henderson, Karaman, Sze, "FSMI: Fast computation of Shannon Mutual Information
 * for information-theoretic mapping" (IJRR 2019). The six variants of Table 1:
 *   FSMI (Theorem 1, Algorithm 1), Approx-FSMI (eq. fsmi_approx, Section 3.4),
 *   Uniform-FSMI (Theorem 4, Algorithm 4), FSMI-RLE (Theorem 3, Algorithm 5),
 *   Approx-FSMI-RLE (Theorem 5, Algorithm 6), Uniform-FSMI-RLE (Theorem 6).
 *
 * Conventions for every entry point:
 *   - Units: one cell (2D) or one virtual cell / voxel (3D) is the unit of length (w = 1).
 *   - Mutual information is returned in nats (natural logarithms), as float32.
 *   - Fixed point: positions are int32 in units of 2^-16 cell (Q16); unit vectors and rotation
 *     entries are int32 in units of 2^-30 (Q30).
 *   - Ownership: every array pointer is device memory owned by the caller (for example a torch
 *     tensor's data_ptr) unless stated otherwise. The library never allocates device memory.
 *   - Asynchrony: work is enqueued on `stream` (NULL = legacy default stream) and the call
 *     returns without waiting. Output arrays are valid once the stream reaches that point.
 *   - Errors: arguments are checked on the host before any launch; on FSMI_ERR_ARG nothing is
 *     launched and outputs are untouched. A launch failure returns FSMI_ERR_CUDA. Conditions only
 *     a kernel can see (a beam longer than its capacity, an RLE output buffer too small) set bits
 *     of a per-device status word that fsmi_device_status() reads; the affected outputs are NaN
 *     (MI) or truncated (runs), never written out of bounds.
 *   - Kernels never wait on other kernels. The only waits inside a kernel are on the CTA's own
 *     tensor-core operations (fsmi_surrogate_predict); each is bounded and, if it gives up, sets
 *     FSMI_STATUS_TIMEOUT and leaves NaN outputs. Nothing here can hang the device.
 *   - Results for a beam whose origin lies outside the map are 0 (the beam crosses no cell).
 */
#ifndef FSMI_H
#define FSMI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared here so the header needs no CUDA include. */
typedef struct CUstream_st *fsmi_stream_t;

typedef enum {
    FSMI_OK = 0,
    FSMI_ERR_ARG = 1,       /* invalid argument: nothing was launched */
    FSMI_ERR_CAPACITY = 2,  /* a size exceeds a documented maximum */
    FSMI_ERR_CUDA = 3,      /* a CUDA runtime call or launch failed */
    FSMI_ERR_TIMEOUT = 4,   /* reserved for bounded device-side waits */
    FSMI_ERR_WORKSPACE = 5  /* the caller's workspace is too small */
} fsmi_status;

typedef enum {
    FSMI_EXACT = 0,   /* Gaussian noise, every cell pair (O(n^2) / O(n_r^2)) */
    FSMI_APPROX = 1,  /* Gaussian truncated to +-trunc_delta cells (O(n Delta) / O(n_r Delta)) */
    FSMI_UNIFORM = 2  /* uniform noise of half-width uniform_h cells (O(n) / O(n_r H)) */
} fsmi_variant;

/* Noise kernel between virtual cells for the RLE variants. Theorem 3 writes G_{k,j} as the
 * Gaussian density at the cell-index distance (FSMI_G_PDF, the default); FSMI_G_ERF uses the
 * Gaussian mass of a unit cell instead, which makes FSMI-RLE on runs equal FSMI on the
 * decompressed cells. */
typedef enum { FSMI_G_PDF = 0, FSMI_G_ERF = 1 } fsmi_kernel;

/* Device status word bits (fsmi_device_status). */
#define FSMI_STATUS_BEAM_OVERFLOW 0x1  /* a beam had more cells than its capacity: its MI is NaN */
#define FSMI_STATUS_RUN_OVERFLOW 0x2   /* RLE output exceeded run_capacity: runs were truncated */
#define FSMI_STATUS_BAD_BEAM 0x4       /* an explicit beam or ray exceeded the per-beam maximum */
#define FSMI_STATUS_INTERNAL 0x8       /* a traversal produced a cell outside the map (library bug) */
#define FSMI_STATUS_TIMEOUT 0x10       /* a bounded wait inside a kernel gave up: its outputs are NaN */

typedef struct {
    int variant;        /* fsmi_variant */
    float sigma;        /* Gaussian range-noise standard deviation, cells, > 0 (EXACT, APPROX) */
    float delta_occ;    /* odds factor for the cell that stops the beam, eq. (inverse_sensing), > 0 */
    float delta_emp;    /* odds factor for cells the beam passed, > 0 */
    int trunc_delta;    /* Delta, cells, >= 0 (APPROX) */
    int uniform_h;      /* H, cells, >= 0 (UNIFORM) */
    float max_range;    /* beam length, cells, in (0, FSMI_MAX_RANGE_2D] (2D); 3D: virtual cells per ray */
    int run_cap;        /* longest run the RLE encoder emits, in [1, 255] */
    int g_kernel;       /* fsmi_kernel (RLE variants) */
    int e0_mode;        /* 2D only: 0 drops the no-return event e_0; 1 places it at virtual index 0
                           (Algorithm 4) with centre l_1 - 1/2 */
    int approx_reading; /* Approx-FSMI-RLE: 0 = Theorem 5's sub-blocks as printed (default),
                           1 = strict band |k - j| <= Delta */
    int flags;          /* FSMI_FLAG_* bits, 0 by default */
} fsmi_params;

/* Exact 2D FSMI evaluates, for each first-hit cell j, the boundary terms of Theorem 1's pair sum
 * within about 5.7 sigma of the cell's centre: every term beyond weighs less than 2^-27 of its
 * factor |C_m - C_{m-1}|, so the MI differs from the full n(n+1) sweep by about one FP32 rounding
 * at most (not bit for bit).
 * FSMI_FLAG_FULL_WINDOW widens the window to every term whose Gaussian tail is non-zero in FP32
 * (about 13.3 sigma; the tail underflows to exactly 0 beyond), which gives the full sweep's result
 * bit for bit; FSMI_FLAG_FULL_SWEEP evaluates all n(n+1) terms (both for verification and timing
 * comparisons). */
#define FSMI_FLAG_FULL_SWEEP 0x1
#define FSMI_FLAG_FULL_WINDOW 0x2

/*
 * Launch schedule of the evaluation kernels, one per kernel family:
 *   FSMI_KIND_2D   fsmi_eval_2d, fsmi_eval_2d_sets, fsmi_eval_beams
 *   FSMI_KIND_RLE  fsmi_eval_rle, fsmi_eval_3d
 * The paper fixes no schedule; this one only changes how beams are dealt to warps and how many
 * warps share a block, never which terms are summed (the RLE cell form below sums the same terms
 * as the run-pair form, in another order). One warp evaluates one beam (or ray) at a time in
 * every schedule; the kernels are persistent (at most as many blocks as fit on the GPU at once).
 * A zero field selects the family's default, given in brackets [2D; RLE].
 */
#define FSMI_KIND_2D 0
#define FSMI_KIND_RLE 1
typedef struct {
    int warps_per_block; /* 1 .. 8 warps per block [4; 2]. Lowered for a call whose per-warp
                            shared arrays would not fit in one block */
    int blocks_per_sm;   /* cap on resident blocks per SM [as many as fit] */
    int queue_chunk;     /* > 0: warps take beams from an atomic work queue, this many consecutive
                            beams per grab, which balances beams of very different lengths; needs
                            a workspace (without one, beams are dealt statically) [1; 4].
                            -1: static grid-stride assignment */
    int cell_runlen;     /* RLE family, variants other than Theorem 5's sub-blocks: a ray whose
                            mean run length is below this is evaluated per virtual cell (a banded
                            convolution, O(n K)) instead of per run pair (O(n_r^2)) [-; 32] */
} fsmi_schedule;

/* Sets the calling thread's schedule of family `kind` (NULL restores the defaults). FSMI_ERR_ARG
 * for an unknown kind or a field out of range. The schedule is read when a call enqueues its
 * kernels. */
fsmi_status fsmi_set_schedule(int kind, const fsmi_schedule *sched);
/* The calling thread's schedule of family `kind`, defaults filled in. */
fsmi_status fsmi_get_schedule(int kind, fsmi_schedule *sched);

/* Documented maxima. */
#define FSMI_MAX_GRID 32767        /* W, H (2D) and X, Y, Z (3D) */
#define FSMI_MAX_RANGE_2D 1024.0f  /* cells; a 2D beam then crosses at most 1451 cells */
#define FSMI_MAX_CELLS 2048        /* cells of one explicit beam (fsmi_eval_beams) */
#define FSMI_MAX_SAMPLES_3D 1024   /* virtual cells of one 3D ray (floor(max_range)) */
#define FSMI_MAX_KERNEL_RADIUS 64  /* RLE noise-kernel support, cells: ceil(7.45 sigma) or H */

/*
 * fsmi_eval_2d - mutual information of every beam of every pose on a 2D occupancy grid.
 * Section 2.4 (problem formulation), Section 3: per beam, the integer fixed-point traversal of
 * the grid gives the ordered cells and their entry distances l_i (l_1 = 0, Section 3.1), then
 * P(e_j) (Algorithm 2), C_k (Algorithm 3) and the variant's pair sum.
 *   map    float32 [H][W] row-major, o in [0, 1] (cell (x, y) at map[y*W + x]).
 *   poses  int32 [P][4]: x, y (Q16, cell units), cos(yaw), sin(yaw) (Q30).
 *   dirs   int32 [B][2]: beam unit vectors in the sensor frame (Q30). Beam b of pose p points
 *          along d = floor((Rot(yaw_p) dirs[b] + 2^29) / 2^30).
 *   out    float32 [P][B], nats.
 *   ws     optional device workspace (NULL allowed), 16-byte aligned. Its first
 *          FSMI_QUEUE_BYTES hold the work-queue counter (fsmi_schedule.queue_chunk). With
 *          fsmi_workspace_size(FSMI_FN_EVAL_2D, W*H) bytes, when the batch visits more cells than
 *          the map holds, the per-cell gains f(delta_occ, r), f(delta_emp, r) are computed once
 *          per map cell (like the paper's look-up table of f, Section 3.3, but exact per cell)
 *          instead of once per visit; the results are the same bit for bit. Calls that share a
 *          workspace must not overlap on the GPU.
 * The traversal is exact integer arithmetic: a cell is entered while its entry distance is
 * < max_range and it lies inside the grid; simultaneous x/y crossings are one diagonal step.
 */
fsmi_status fsmi_eval_2d(const float *map, int W, int H, const int32_t *poses, int P,
                         const int32_t *dirs, int B, const fsmi_params *prm, float *out,
                         void *ws, size_t ws_bytes, fsmi_stream_t stream);

/*
 * fsmi_eval_2d_sets - fsmi_eval_2d over several candidate sets in one launch: each set has its
 * own poses, beam directions, beam count and range (beams of very different lengths, Table 1's
 * O(n^2) cost per beam, share one persistent kernel; pair it with a work queue).
 *   poses  int32 [P][4], dirs int32 [B][2]: as fsmi_eval_2d; sets index into them.
 *   sets   device array of nsets descriptors (below), in increasing beam_offset order with
 *          sets[0].beam_offset = 0 and beam_offset[s+1] = beam_offset[s] + npose[s] * nbeam[s];
 *          nbeams = the sum of npose * nbeam.
 *   prm    as fsmi_eval_2d; prm->max_range bounds every set's max_range (it sizes the per-beam
 *          capacity).
 *   out    float32 [nbeams]: out[beam_offset + p * nbeam + b] for pose p and beam b of a set.
 *   ws     as fsmi_eval_2d (workspace size from fsmi_workspace_size(FSMI_FN_EVAL_2D, W*H)).
 * The descriptors live in device memory and are checked by the kernel: a beam whose set indexes
 * past P or B, has a max_range outside (0, prm->max_range], or is not covered by its set, gets NaN
 * and sets FSMI_STATUS_BAD_BEAM.
 */
typedef struct {
    int pose_offset;       /* first pose of the set in `poses` */
    int npose;             /* poses in the set, >= 0 */
    int dir_offset;        /* first beam direction of the set in `dirs` */
    int nbeam;             /* beams per pose, >= 0 */
    float max_range;       /* beam length of this set, cells */
    int reserved;          /* 0 */
    long long beam_offset; /* first output index of the set */
} fsmi_set_2d;

fsmi_status fsmi_eval_2d_sets(const float *map, int W, int H, const int32_t *poses, int P,
                              const int32_t *dirs, int B, const fsmi_set_2d *sets, int nsets,
                              long long nbeams, const fsmi_params *prm, float *out, void *ws,
                              size_t ws_bytes, fsmi_stream_t stream);

/*
 * fsmi_eval_mixed - a stream of candidate sets of both kinds in one persistent launch: 2D sets
 * (beams on the occupancy grid, as fsmi_eval_2d) and 3D sets (rays through voxel submaps,
 * sampled, run-length encoded and evaluated as fsmi_eval_3d). The sets form one ordered list of
 * work items (one beam or ray each), taken by the warps in list order through the work queue, so
 * sets complete roughly in the order given.
 *   map, W, H, poses2 [P2][4], dirs2 [B2][2], prm2: the 2D part (prm2 NULL if there is no 2D set);
 *     prm2->max_range bounds the sets' beam lengths.
 *   vols [nvol] (device array of fsmi_volume), poses3 [P3][12], dirs3 [R3][3], prm3: the 3D part
 *     (prm3 NULL if there is no 3D set); prm3->max_range bounds the sets' virtual cells per ray.
 *   sets [nsets] (device array), sorted by out_offset, contiguous: out_offset[0] = 0,
 *     out_offset[s+1] = out_offset[s] + npose[s] * ndir[s]; nitems = the total.
 *   out float32 [nitems]: out[out_offset + p * ndir + d] in nats.
 *   times (optional) uint64 [nitems + 1]: times[0] = the earliest block start, times[1 + i] = the
 *     %globaltimer value (ns) when item i finished; a set's latency is the largest of its items'
 *     times minus times[0].
 *   ws: 16-byte aligned; fsmi_workspace_size(FSMI_FN_EVAL_2D, W*H) bytes (queue counter and 2D
 *     per-cell gains), or FSMI_QUEUE_BYTES without 2D sets. With fsmi_mixed_workspace_size(W*H
 *     (0 without 2D sets), nsets) bytes the call also plans by range class: a one-warp pre-pass
 *     lists the sets, in stream order, by kind and range class (16 classes per kind, bounds from
 *     16 to 1024 cells about a factor 1.25 apart), and each class runs as its own persistent launch whose warps' shared arrays are sized
 *     for that class rather than for the stream's longest beam; the classes run one after the
 *     other, in that order. Results are the same floats either way. If any descriptor fails the
 *     plan's checks (those below, and outputs contiguous in set order) the single launch runs.
 * Descriptors are checked per item in the kernel: an item of a malformed set (indices past the
 * pose or direction arrays, a range outside its bound, a kind without parameters, a volume index
 * outside [0, nvol)) gets NaN and sets FSMI_STATUS_BAD_BEAM. The work schedule is the 2D family's.
 */
#define FSMI_SET_2D 0
#define FSMI_SET_3D 1
typedef struct {
    const float *vox; /* float32 [Z][Y][X] voxel occupancy, device memory */
    int X, Y, Z;
    int reserved;     /* 0 */
} fsmi_volume;

typedef struct {
    int kind;              /* FSMI_SET_2D or FSMI_SET_3D */
    int pose_offset;       /* first pose of the set in its kind's pose array */
    int npose;             /* poses, >= 0 */
    int dir_offset;        /* first direction in its kind's direction array */
    int ndir;              /* beams (rays) per pose, >= 1 */
    float max_range;       /* 2D: beam length, cells; 3D: virtual cells per ray (its floor) */
    int volume;            /* 3D: index into vols */
    int reserved;          /* 0 */
    long long out_offset;  /* first output index */
} fsmi_set;

fsmi_status fsmi_eval_mixed(const float *map, int W, int H, const int32_t *poses2, int P2,
                            const int32_t *dirs2, int B2, const fsmi_params *prm2,
                            const fsmi_volume *vols, int nvol, const int32_t *poses3, int P3,
                            const int32_t *dirs3, int R3, const fsmi_params *prm3, const fsmi_set *sets,
                            int nsets, long long nitems, float *out, unsigned long long *times, void *ws,
                            size_t ws_bytes, fsmi_stream_t stream);

/* Workspace bytes of fsmi_eval_mixed with the range-class plan: the queue counter, 16 bytes of
 * gains per map cell (map_cells = W*H, or 0 without 2D sets) and the plan for nsets sets. */
fsmi_status fsmi_mixed_workspace_size(long long map_cells, int nsets, size_t *bytes);

/*
 * fsmi_eval_beams - the same pair sums on explicit beams (Theorem 1's inputs: o_i, l_i).
 *   off    int32 [nbeams+1] CSR offsets; beam b owns cells off[b] .. off[b+1]-1
 *          (at most FSMI_MAX_CELLS cells).
 *   o      float32 [off[nbeams]] occupancy probabilities, in beam order.
 *   l      float32 [off[nbeams]] entry distances, increasing within a beam, first one 0.
 *   lend   float32 [nbeams] end distance l_{n+1} of each beam.
 *   out    float32 [nbeams], nats.
 *   ws     optional workspace of FSMI_QUEUE_BYTES (16-byte aligned) for the work queue.
 */
fsmi_status fsmi_eval_beams(const int32_t *off, const float *o, const float *l, const float *lend,
                            int nbeams, const fsmi_params *prm, float *out, void *ws,
                            size_t ws_bytes, fsmi_stream_t stream);

/*
 * fsmi_trace_2d - exports the traversal used by fsmi_eval_2d (same inputs) so that cell lists
 * can be compared bit for bit.
 *   cells  int32 [P*B][cap]: cell ids y*W + x in beam order.
 *   l      float32 [P*B][cap+1]: entry distances, then the end distance at index n.
 *   n      int32 [P*B]: cell count, or -1 if the beam has more than cap cells.
 */
fsmi_status fsmi_trace_2d(int W, int H, const int32_t *poses, int P, const int32_t *dirs, int B,
                          float max_range, int cap, int32_t *cells, float *l, int32_t *n,
                          fsmi_stream_t stream);

/*
 * fsmi_rle_encode_3d - Section 4: each ray is projected onto equal virtual cells (cell i is the
 * voxel holding o + (i + 1/2) d, i = 0 .. floor(max_range)-1, stopping at the grid boundary),
 * and the occupancy sequence is run-length encoded (eq. occup_rle) into maximal runs of
 * bit-identical values, split greedily from the sensor into runs of at most run_cap cells.
 *   vox      float32 [Z][Y][X], o in [0, 1] (voxel (x, y, z) at vox[(z*Y + y)*X + x]).
 *   poses    int32 [P][12]: x, y, z (Q16), then the sensor rotation R row-major (Q30).
 *   dirs     int32 [R][3]: ray unit vectors in the sensor frame (Q30); ray r of pose p points
 *            along d = floor((R_p dirs[r] + 2^29) / 2^30).
 *   run_off  int32 [P*R+1] output CSR offsets (ray i = p*R + r).
 *   run_o    float32 [run_capacity], run_len uint8 [run_capacity]: output runs.
 *   ws       device workspace of at least fsmi_workspace_size(FSMI_FN_RLE_ENCODE_3D, ...) bytes.
 * If the runs exceed run_capacity, the status bit FSMI_STATUS_RUN_OVERFLOW is set, run_off
 * still holds the full offsets and only runs below run_capacity are written. The offsets are
 * int32: where the runs of a batch pass INT32_MAX in total, the offsets beyond saturate at
 * INT32_MAX (never wrap) and FSMI_STATUS_RUN_OVERFLOW is set.
 */
fsmi_status fsmi_rle_encode_3d(const float *vox, int X, int Y, int Z, const int32_t *poses, int P,
                               const int32_t *dirs, int R, const fsmi_params *prm, int32_t *run_off,
                               float *run_o, uint8_t *run_len, int run_capacity, void *ws,
                               size_t ws_bytes, fsmi_stream_t stream);

/*
 * fsmi_rle_encode_3d_noalloc - fsmi_rle_encode_3d for callers that cannot allocate device memory
 * when they encode (for example a planner inside a real-time control loop whose device memory is
 * reserved up front, or code that is handed only input and output pointers). The paper has no
 * counterpart: this is a library convenience, not part of the method.
 *   Arguments and results are those of fsmi_rle_encode_3d without the workspace: the offset scan
 *   keeps its tile totals in a 16 KiB array owned by the library, which every GPU that loads the
 *   library holds until the process exits. Nothing is allocated and no allocating routine is
 *   called.
 *   At most FSMI_NOALLOC_MAX_RAYS rays (P*R) per call; more returns FSMI_ERR_CAPACITY and launches
 *   nothing.
 *   The first call on each device looks up the array's device address (with that device
 *   current); make that first call before capturing a stream.
 *   All calls share the one array: calls whose work overlaps on the GPU (different streams, or
 *   different host threads on the same device) race and must be serialised by the caller. Each
 *   call overwrites every entry it reads, so no clearing is needed between calls.
 */
#define FSMI_NOALLOC_MAX_RAYS (4096LL * 4096LL)
fsmi_status fsmi_rle_encode_3d_noalloc(const float *vox, int X, int Y, int Z, const int32_t *poses,
                                       int P, const int32_t *dirs, int R, const fsmi_params *prm,
                                       int32_t *run_off, float *run_o, uint8_t *run_len,
                                       int run_capacity, fsmi_stream_t stream);

/*
 * fsmi_eval_rle - FSMI-RLE (Theorem 3), Approx-FSMI-RLE (Theorem 5) or Uniform-FSMI-RLE
 * (Theorem 6) of run-length-encoded rays.
 *   run_off  int32 [nrays+1] CSR offsets; ray r owns runs run_off[r] .. run_off[r+1]-1 whose
 *            lengths sum to at most FSMI_MAX_SAMPLES_3D virtual cells.
 *   run_o    float32 occupancy of each run; run_len uint8 length (>= 1) of each run.
 *   out      float32 [nrays], nats.
 *   ws       optional workspace of FSMI_QUEUE_BYTES (16-byte aligned) for the work queue.
 */
fsmi_status fsmi_eval_rle(const int32_t *run_off, const float *run_o, const uint8_t *run_len,
                          int nrays, const fsmi_params *prm, float *out, void *ws, size_t ws_bytes,
                          fsmi_stream_t stream);

/*
 * fsmi_eval_3d - fused 3D path: sampling, run-length encoding and the RLE variant of every ray,
 * with the runs kept on chip. Same inputs as fsmi_rle_encode_3d; out float32 [P][R] in nats;
 * nruns (optional, may be NULL) int32 [P][R] receives each ray's run count; ws optional
 * workspace of FSMI_QUEUE_BYTES (16-byte aligned) for the work queue.
 */
fsmi_status fsmi_eval_3d(const float *vox, int X, int Y, int Z, const int32_t *poses, int P,
                         const int32_t *dirs, int R, const fsmi_params *prm, float *out,
                         int32_t *nruns, void *ws, size_t ws_bytes, fsmi_stream_t stream);

/*
 * fsmi_gauss_tail - the library's Gaussian tail, exposed so its accuracy can be tested:
 *   out[i] = 0.5 * erfc(s[i] / sqrt(log2 e)) for s[i] >= 0 (float32, device arrays of n).
 * The pair sums of the Gaussian variants (Theorem 1, eq. fsmi_approx) evaluate
 * G_{k,j} = Phi(x_{k+1}) - Phi(x_k) through this tail. Absolute error <= 3e-7; <= 4e-6 of the
 * value plus 6e-8 everywhere.
 */
fsmi_status fsmi_gauss_tail(const float *s, float *out, long long n, fsmi_stream_t stream);

/*
 * fsmi_probe - measurement kernels for the rooflines of the kernels above (not part of the
 * method; the paper has no counterpart). One launch on `stream`; the caller times it with CUDA
 * events and divides the work by the time:
 *   FSMI_PROBE_EX2, _RCP, _FMA, _FMA2: fsmi_probe_threads(probe) threads each run iters x 8
 *     dependent ex2.approx.ftz.f32 / rcp.approx.ftz.f32 (+ one add.f32 each) / fma.rn.f32 /
 *     fma.rn.f32x2 instructions (eight independent chains). buf: >= 4 bytes, never written in
 *     practice (a sink that keeps the work alive).
 *   FSMI_PROBE_READ: iters passes over the bytes of buf (16-byte aligned, a multiple of 16), each
 *     a grid-strided float4 read cached in L2 only: L2 read bandwidth for a buffer well inside L2,
 *     HBM read bandwidth for one several times larger.
 *   FSMI_PROBE_SPIN: one warp spins for iters SM clock cycles (<= 2^40) and stores the cycle
 *     count in buf (int64, 8-byte aligned): the SM clock is iters / the launch's duration.
 * Returns FSMI_ERR_ARG for an unknown probe or a buffer that does not fit.
 */
#define FSMI_PROBE_EX2 0
#define FSMI_PROBE_RCP 1
#define FSMI_PROBE_FMA 2
#define FSMI_PROBE_FMA2 3
#define FSMI_PROBE_READ 4
#define FSMI_PROBE_SPIN 5
fsmi_status fsmi_probe(int probe, long long iters, void *buf, size_t bytes, fsmi_stream_t stream);
/* threads of one fsmi_probe launch of `probe` on the current device (0 if unknown) */
int fsmi_probe_threads(int probe);

/*
 * The exploration loop around the beam MI (Section 2.4; eq. (1) of Section 2.1).
 *
 * fsmi_eval_trajectories_2d - mutual information along discretised candidate trajectories: the
 * MI of a trajectory is the sum over its states of the scan MI (the sum of the state's beam MI),
 * where a cell that already contributed at an earlier state of the same trajectory adds nothing
 * (it keeps its occupancy, so it still stops the beam with probability o, but its terms
 * f(delta, r) leave C_k). The beams of one state are summed as a scan, without marks between
 * them. Trajectories are independent of one another.
 *   poses     int32 [P][4] as fsmi_eval_2d: every state of every trajectory.
 *   traj_off  int32 [T+1] device CSR offsets: trajectory t has states traj_off[t] ..
 *             traj_off[t+1]-1 in travel order (traj_off[0] = 0, traj_off[T] = P, non-decreasing);
 *             a pose outside every trajectory gets NaN beams and FSMI_STATUS_BAD_BEAM.
 *   dirs, B, prm, map: as fsmi_eval_2d.
 *   beam_mi   float32 [P][B] (device, output), state_mi float32 [P], traj_mi float32 [T].
 *   ws        required, 16-byte aligned, fsmi_trajectory_workspace_size(W, H, T) bytes: the
 *             queue counter, per-map-cell gains and one int32 visit stamp per map cell and
 *             trajectory (the first state whose beams cross the cell).
 * Sums are taken in a fixed order, so results do not change from run to run.
 */
fsmi_status fsmi_trajectory_workspace_size(int W, int H, int T, size_t *bytes);
fsmi_status fsmi_eval_trajectories_2d(const float *map, int W, int H, const int32_t *poses, int P,
                                      const int32_t *traj_off, int T, const int32_t *dirs, int B,
                                      const fsmi_params *prm, float *beam_mi, float *state_mi,
                                      float *traj_mi, void *ws, size_t ws_bytes,
                                      fsmi_stream_t stream);

/* fsmi_best_trajectory - the trajectory with the most mutual information per travel distance
 * (Sections 2.4 and 5.2): ratio[t] = traj_mi[t] / max(1, L_t), L_t the sum of the straight
 * distances (cells) between consecutive states (poses int32 [P][4], traj_off as above; offsets are
 * clamped to [0, P]); *best (device int32) = argmax of ratio, the lowest index among equal ratios,
 * -1 if none is a number. T >= 1. */
fsmi_status fsmi_best_trajectory(const float *traj_mi, const int32_t *poses, int P,
                                 const int32_t *traj_off, int T, float *ratio, int32_t *best,
                                 fsmi_stream_t stream);

/* fsmi_scan_sums - pose_mi[p] = sum over b of beam_mi[p*B + b] (the scan MI of each candidate
 * pose), in a fixed order. */
fsmi_status fsmi_scan_sums(const float *beam_mi, long long P, int B, float *pose_mi,
                           fsmi_stream_t stream);

/*
 * fsmi_update_map_2d - the Bayesian occupancy update of eq. (1) with the inverse sensor model of
 * Section 2.2, for a batch of measured beams: the odds of the cell where a measured range ends are
 * multiplied by delta_occ, those of every cell the beam crossed before it by delta_emp, the rest
 * are unchanged. The traversal is fsmi_eval_2d's cut at the measured range, so the cell holding
 * the range end is decided exactly (its entry distance is below the range, the next one is not).
 *   map     float32 [H][W], updated in place; cells at exactly 0 or 1 stay put.
 *   poses, dirs: as fsmi_eval_2d; ranges float32 [P][B] measured range per beam, cells. A range
 *           >= prm->max_range (or +inf) is a beam without return: every cell up to max_range is
 *           crossed (delta_emp). A range that is NaN or <= 0 is no measurement. A range that ends
 *           outside the grid updates only the cells crossed inside it.
 *   prm     delta_occ, delta_emp, max_range (other fields must be valid but are not used).
 *   ws      16-byte aligned, fsmi_workspace_size(FSMI_FN_UPDATE_MAP_2D, W*H) bytes (per-cell
 *           update counts).
 * Updates commute, so the batch is applied at once per cell as
 * o' = 1 / (1 + exp(-(logit(o) + a ln delta_occ + b ln delta_emp))) with a, b the cell's counts.
 */
fsmi_status fsmi_update_map_2d(float *map, int W, int H, const int32_t *poses, int P,
                               const int32_t *dirs, int B, const float *ranges,
                               const fsmi_params *prm, void *ws, size_t ws_bytes,
                               fsmi_stream_t stream);

/*
 * Learned surrogate (not part of the paper; a library extension that prescreens candidate poses
 * before exact FSMI reranks the best of them). One 2D beam's occupancy profile -> its predicted MI:
 *   input  x[256][2]: sample i at distance i + 1/2 cells along the beam (the cell holding
 *          o + (i + 1/2) d, d the beam's Q30 direction); (o, 1) inside the map, (0, 0) beyond it
 *   conv1  2 -> 32 channels, kernel 3, stride 2, zero padding 1, ReLU (256 -> 128 positions);
 *   conv2, conv3  32 -> 32, the same (-> 64 -> 32); fc1 1024 -> 256 (input t * 32 + c), ReLU;
 *   fc2 256 -> 1.   conv: z[t][c] = b[c] + sum_{k<3} sum_ci W[c][k][ci] a[2t + k - 1][ci].
 * Parameters: one flat float32 vector of FSMI_SURR_NPARAMS in the order W1 [32][3][2], b1 [32],
 * W2 [32][3][32], b2, W3 [32][3][32], b3, W4 [256][1024], b4 [256], W5 [256], b5 [1]. Compute uses
 * a BF16 copy of the same vector for the weights (uint16 bit patterns) and the float32 biases,
 * with FP32 accumulation.
 */
#define FSMI_SURR_L 256
#define FSMI_SURR_NPARAMS 269089

/* fsmi_profiles_2d - BF16 profiles out [N][256][2] of beams `beam_ids` (flat p * B + b; NULL = all
 * N = P * B beams in order). An id outside [0, P * B) gives an all-zero profile and sets
 * FSMI_STATUS_BAD_BEAM. max_range (cells): a sample at distance i + 1/2 >= max_range reads as
 * outside the map, (0, 0), as if the map ended there (a beam cut at range R crosses the same cells
 * as one whose map ends at R); max_range <= 0 keeps all 256 samples. NaN is an argument error. */
fsmi_status fsmi_profiles_2d(const float *map, int W, int H, const int32_t *poses, int P,
                             const int32_t *dirs, int B, float max_range, const int32_t *beam_ids,
                             long long N, uint16_t *out, fsmi_stream_t stream);

/* Workspace of fsmi_surrogate_loss_grad for a batch of N (mode 0) or of fsmi_surrogate_predict
 * for N beams (mode 1). */
fsmi_status fsmi_surrogate_workspace_size(int mode, long long N, size_t *bytes);

/* fsmi_surrogate_loss_grad - one training step's forward and backward on a batch of N profiles
 * x [N][256][2] (BF16) with targets y [N]: loss = mean (pred - y)^2 (device float) and its gradient
 * grad [FSMI_SURR_NPARAMS] with respect to the parameters (through the BF16 weights). Activations
 * are kept in FP32; the layers' products run on the tensor cores with each FP32 operand split into
 * BF16 terms (three in the forward pass, as accurate as FP32 arithmetic; two in the backward
 * pass). pred (optional) receives the N predictions. On return the workspace begins with the FP32
 * pre-activations z1 [N][128][32], z2 [N][64][32], z3 [N][32][32], z4 [N][256], in that order.
 * 1 <= N <= 65536. Deterministic. */
fsmi_status fsmi_surrogate_loss_grad(const float *params, const uint16_t *wbf16, const uint16_t *x,
                                     const float *y, int N, float *grad, float *loss, float *pred,
                                     void *ws, size_t ws_bytes, fsmi_stream_t stream);

/* fsmi_surrogate_adam - one Adam step (Kingma and Ba) with bias correction at step t >= 1 on params,
 * moments m, v (all float32 [FSMI_SURR_NPARAMS]); refreshes the BF16 copy wbf16.
 * fsmi_surrogate_cast - wbf16 = BF16(params) (round to nearest even). */
fsmi_status fsmi_surrogate_adam(float *params, float *m, float *v, const float *grad, float lr,
                                float beta1, float beta2, float eps, int t, uint16_t *wbf16,
                                fsmi_stream_t stream);
fsmi_status fsmi_surrogate_cast(const float *params, uint16_t *wbf16, fsmi_stream_t stream);

/* fsmi_surrogate_predict - predictions pred [P*B] for every beam of every pose on the map (the
 * profiles are sampled inside the kernel, cut at max_range as in fsmi_profiles_2d), or, with
 * map == NULL, for N given profiles x (max_range unused). The conv layers (mma.sync) and fc1
 * (tcgen05, accumulators in TMEM) run on the tensor cores with BF16 activations between layers and
 * FP32 accumulation; fc2 reads the fc1 activations in FP32.
 * ws: fsmi_surrogate_workspace_size(1, N) bytes, 16-byte aligned. */
fsmi_status fsmi_surrogate_predict(const float *params, const uint16_t *wbf16, const float *map,
                                   int W, int H, const int32_t *poses, int P, const int32_t *dirs,
                                   int B, float max_range, const uint16_t *x, long long N, float *pred,
                                   void *ws, size_t ws_bytes, fsmi_stream_t stream);

/* fsmi_topk - idx [k] = indices of the k largest of v [n] in descending order, lower index first
 * among equal values, NaN last. 1 <= k <= n <= 16384. */
fsmi_status fsmi_topk(const float *v, int n, int k, int32_t *idx, fsmi_stream_t stream);

/* fsmi_gather_rows - dst[r][.] = src[idx[r]][.] for k rows of `width` int32 out of src's nrows
 * (e.g. the poses a prescreen selected); an index outside [0, nrows) gives a row of zeros and sets
 * FSMI_STATUS_BAD_BEAM. */
fsmi_status fsmi_gather_rows(const int32_t *src, long long nrows, int width, const int32_t *idx, int k,
                             int32_t *dst, fsmi_stream_t stream);

/* Function ids for fsmi_workspace_size. */
#define FSMI_FN_EVAL_2D 0
#define FSMI_FN_EVAL_BEAMS 1
#define FSMI_FN_RLE_ENCODE_3D 2
#define FSMI_FN_EVAL_RLE 3
#define FSMI_FN_EVAL_3D 4
#define FSMI_FN_UPDATE_MAP_2D 5

/* Bytes at the front of an evaluation workspace that hold the work-queue counter. */
#define FSMI_QUEUE_BYTES 256

/* Bytes of device workspace entry point `fn` can use for `nitems` items: map cells for
 * FSMI_FN_EVAL_2D (queue counter + optional gains; also fsmi_eval_2d_sets), rays for
 * FSMI_FN_RLE_ENCODE_3D (required offset scan), map cells for FSMI_FN_UPDATE_MAP_2D (required
 * update counts), FSMI_QUEUE_BYTES for the other evaluations. */
fsmi_status fsmi_workspace_size(int fn, long long nitems, const fsmi_params *prm, size_t *bytes);

/*
 * Native schedule tuning and CUDA-graph helpers (library conveniences; the paper has none).
 *
 * fsmi_autotune - times `fn(ctx, stream)` (which makes one or more fsmi_* calls of family `kind`
 * on `stream`) under each of the ncands schedules of that family: one untimed call, then `reps`
 * calls between two CUDA events. On return the calling thread's schedule of that family is the
 * fastest one, copied to *best with defaults filled in; ms (optional, host float [ncands])
 * receives each candidate's mean milliseconds per call, or -1 where fn failed. FSMI_ERR_ARG if
 * every candidate failed (the schedule is then left as it was). fn must not capture or
 * synchronise other streams.
 */
typedef fsmi_status (*fsmi_tune_fn)(void *ctx, fsmi_stream_t stream);
fsmi_status fsmi_autotune(int kind, fsmi_tune_fn fn, void *ctx, const fsmi_schedule *cands,
                          int ncands, int reps, fsmi_stream_t stream, fsmi_schedule *best,
                          float *ms);

/* Default candidate schedules of family `kind` for fsmi_autotune, every field filled in as
 * fsmi_get_schedule reports them: FSMI_KIND_2D 2, 4, 8 warps x chunk 1, 4, static (9);
 * FSMI_KIND_RLE 1, 2, 4 warps x chunk 2, 4, 8, static x cell_runlen 16, 32 (24). Writes at most
 * `max` entries to out (host) and their number to *n. */
fsmi_status fsmi_schedule_candidates(int kind, fsmi_schedule *out, int max, int *n);

/* Does every per-device lookup and kernel load of the library on the current device, so that
 * fsmi_* calls can then be captured into a CUDA graph. */
fsmi_status fsmi_prepare(void);

/* Stream capture of fsmi_* calls into a replayable graph. `stream` must not be the legacy
 * default stream (NULL). Between begin and end, make only asynchronous calls on `stream`
 * (fsmi_device_status synchronises and is not allowed). Workspace queue counters are reset by a
 * captured memset, so a graph can be replayed any number of times; replays of one graph, or of
 * graphs sharing a workspace, must not overlap on the GPU. */
typedef struct fsmi_graph_st *fsmi_graph;
fsmi_status fsmi_capture_begin(fsmi_stream_t stream);
fsmi_status fsmi_capture_end(fsmi_stream_t stream, fsmi_graph *graph);
fsmi_status fsmi_graph_launch(fsmi_graph graph, fsmi_stream_t stream);
fsmi_status fsmi_graph_destroy(fsmi_graph graph);

/* Poll limit, for the calling host thread, of the one device-side wait a caller can shorten: the
 * surrogate inference kernel's epilogue waiting for its tensor-core accumulator
 * (fsmi_surrogate_predict). polls >= 0 sets it, < 0 restores the default (2^22 polls, far longer
 * than the tensor cores take). A limit too short for the MMAs makes that wait give up: the call
 * then sets FSMI_STATUS_TIMEOUT, writes NaN predictions, and still returns only after its copies
 * and MMAs in flight have completed (those waits keep the full limit), so the device stays usable.
 * It exists so that the timeout path can be tested without faulting or hanging the GPU; the paper
 * has no counterpart. */
fsmi_status fsmi_set_wait_limit(long long polls);

/* Waits for `stream`, then returns in *status the current device's status word (FSMI_STATUS_*
 * bits, 0 if clean) and clears it. *status is host memory. */
fsmi_status fsmi_device_status(fsmi_stream_t stream, int *status);

/* Human-readable name of a status code (static string). */
const char *fsmi_status_str(fsmi_status s);

/* The cudaError_t value behind the calling thread's last FSMI_ERR_CUDA (0 if none). */
int fsmi_last_cuda_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int fsmi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FSMI_H */
