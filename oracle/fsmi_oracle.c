/*
 * FP64 CPU oracle for FSMI: Zhang, Henderson, Karaman, Sze, "FSMI: Fast computation of Shannon
 * Mutual Information for information-theoretic mapping" (IJRR 2019).
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously-correct reference that the CUDA
 * library is checked against. Only the tests, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py may load it. It shares no code, header, table or helper with the CUDA library; the two
 * meet only at the seeded input arrays.
 *
 * Every quantity is computed in double precision by the definition the paper gives, in the
 * paper's order; library primitives (erfc, exp, log, log1p, pow) are the only building blocks.
 * No blocking, fusion, telescoping or reordering beyond what the cited equation states.
 *
 * Conventions (readings of passages the paper leaves open or states ambiguously):
 *   - natural logarithms: mutual information is in nats;
 *   - cells are 0-based here: paper cell i (1..n) is index i-1; boundaries l[0..n] with l[0] = l_1 = 0;
 *   - the no-return event e_0 is dropped by default (e0_mode = 0); e0_mode = 1 places it at the
 *     virtual index 0 used by Algorithm 4, with a Gaussian centred at l_1 - w/2 (w = 1 cell);
 *   - a measurement outside [l_1, l_{n+1}) carries no information (Theorem 1 sums k = 1..n).
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EXPORT __attribute__((visibility("default")))

enum { OV_EXACT = 0, OV_APPROX = 1, OV_UNIFORM = 2 };
enum { OG_PDF = 0, OG_ERF = 1 };

struct oracle_params {
    int variant;        /* OV_EXACT, OV_APPROX (Gaussian truncated to +-trunc_delta cells), OV_UNIFORM */
    double sigma;       /* range-noise standard deviation, in cells */
    double delta_occ;   /* inverse sensor model odds factors, Section 2.2 */
    double delta_emp;
    int trunc_delta;    /* Delta of Approx-FSMI / Approx-FSMI-RLE, in cells */
    int uniform_h;      /* H of Uniform-FSMI / Uniform-FSMI-RLE, in cells */
    double max_range;   /* beam length limit, in cells */
    int run_cap;        /* longest run the RLE encoder emits */
    int g_kernel;       /* RLE noise kernel between virtual cells: OG_PDF (Theorem 3 as printed) or OG_ERF */
    int e0_mode;        /* 0: drop e_0; 1: Algorithm-4 placement (2D variants only) */
    int approx_reading; /* Approx-FSMI-RLE: 0 = Theorem 5 sub-blocks as printed, 1 = strict band |k-j| <= Delta */
};

/* ------------------------------------------------------------------------------------------ */
/* Section 2.2: per-cell information gain f(delta, r)                                          */
/* ------------------------------------------------------------------------------------------ */

/* f(delta, r) = log((r+1)/(r+1/delta)) - log(delta)/(r delta + 1), as printed (odds form). */
ORACLE_EXPORT double oracle_f_odds(double delta, double r)
{
    return log((r + 1.0) / (r + 1.0 / delta)) - log(delta) / (r * delta + 1.0);
}

/* The same function written in the occupancy probability o = r/(1+r), finite at o in {0, 1}:
 * with a = o(delta-1), f = log(delta) * o*delta/(1+a) - log(1+a). */
ORACLE_EXPORT double oracle_f_prob(double delta, double o)
{
    double a = o * (delta - 1.0);
    return log(delta) * o * delta / (1.0 + a) - log1p(a);
}

/* ------------------------------------------------------------------------------------------ */
/* Algorithm 2: first-hit probabilities; Algorithm 3: C_k                                      */
/* ------------------------------------------------------------------------------------------ */

/* pe[0] = P(e_0) = prod (1-o_l); pe[j] = P(e_j) = E_{j-1} o_j for paper cells j = 1..n. */
ORACLE_EXPORT void oracle_first_hit(const double *o, int n, double *pe)
{
    double E = 1.0;
    for (int j = 1; j <= n; ++j) {
        pe[j] = E * o[j - 1];
        E = E * (1.0 - o[j - 1]);
    }
    pe[0] = E;
}

/* C[k-1] = C_k = q_{k-1} + f(delta_occ, r_k), q_k = q_{k-1} + f(delta_emp, r_k), k = 1..n. */
ORACLE_EXPORT void oracle_c_k(const double *o, int n, double docc, double demp, double *C)
{
    double q = 0.0;
    for (int k = 1; k <= n; ++k) {
        C[k - 1] = q + oracle_f_prob(docc, o[k - 1]);
        q = q + oracle_f_prob(demp, o[k - 1]);
    }
}

static double Phi(double x) { return 0.5 * erfc(-x / M_SQRT2); }

/* ------------------------------------------------------------------------------------------ */
/* 2D variants on one explicit beam: o[n], l[n+1] (l[0] = 0, increasing)                       */
/* ------------------------------------------------------------------------------------------ */

/* G_{k,j} of Section 3.3 (Lemma on Phi): Gaussian mass of cell k for a beam stopped in cell j.
 * k, j are paper indices; j = 0 is the e_0 placement with centre l_1 - 1/2. */
static double G_gauss(const double *l, int k, int j, double sigma)
{
    double mu = (j == 0) ? (l[0] - 0.5) : 0.5 * (l[j - 1] + l[j]);
    return Phi((l[k] - mu) / sigma) - Phi((l[k - 1] - mu) / sigma);
}

/* C_k of a beam some of whose cells are excluded from the sum of eq. (mi_sum) (Section 2.4: cells
 * that already contributed along a trajectory add nothing): an excluded cell keeps its occupancy
 * (it still stops the beam) but its terms f(delta_occ, r_k), f(delta_emp, r_k) are dropped.
 * skip = NULL excludes nothing (then this is Algorithm 3). */
static void c_k_skip(const double *o, const unsigned char *skip, int n, double docc, double demp, double *C)
{
    double q = 0.0;
    for (int k = 1; k <= n; ++k) {
        int use = !(skip && skip[k - 1]);
        C[k - 1] = q + (use ? oracle_f_prob(docc, o[k - 1]) : 0.0);
        q = q + (use ? oracle_f_prob(demp, o[k - 1]) : 0.0);
    }
}

/* FSMI (Theorem 1 / Algorithm 1), Approx-FSMI (eq. fsmi_approx) and Uniform-FSMI (Theorem 4 /
 * Algorithm 4) for one beam, summing the cells not excluded by skip (NULL: all cells). */
ORACLE_EXPORT double oracle_fsmi_beam_skip(const double *o, const double *l, const unsigned char *skip, int n,
                                           const struct oracle_params *p)
{
    if (n <= 0) return 0.0;
    double *pe = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *C = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    oracle_first_hit(o, n, pe);
    c_k_skip(o, skip, n, p->delta_occ, p->delta_emp, C);
    int j0 = p->e0_mode ? 0 : 1;
    double I = 0.0;
    if (p->variant == OV_EXACT || p->variant == OV_APPROX) {
        for (int j = j0; j <= n; ++j) {
            int klo = 1, khi = n;
            if (p->variant == OV_APPROX) {
                if (j - p->trunc_delta > klo) klo = j - p->trunc_delta;
                if (j + p->trunc_delta < khi) khi = j + p->trunc_delta;
            }
            for (int k = klo; k <= khi; ++k)
                I += pe[j] * C[k - 1] * G_gauss(l, k, j, p->sigma);
        }
    } else {
        /* Algorithm 4: D_k = sum_{i<=k} C_i, D_0 = 0, indices clamped to [0, n]. */
        double *D = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        D[0] = 0.0;
        for (int k = 1; k <= n; ++k) D[k] = D[k - 1] + C[k - 1];
        int H = p->uniform_h;
        for (int j = j0; j <= n; ++j) {
            int hi = j + H < n ? j + H : n;
            int lo = j - H - 1 > 0 ? j - H - 1 : 0;
            I += pe[j] * (D[hi] - D[lo]) / (2.0 * H + 1.0);
        }
        free(D);
    }
    free(pe);
    free(C);
    return I;
}

ORACLE_EXPORT double oracle_fsmi_beam(const double *o, const double *l, int n, const struct oracle_params *p)
{
    return oracle_fsmi_beam_skip(o, l, NULL, n, p);
}

/* Uniform-FSMI as the generic pair sum of eq. (uniform): sum_j P(e_j) sum_k C_k G^U_{k,j}, with
 * G^U_{k,j} the mass that U[l_j - H, l_{j+1} + H] puts on [l_k, l_{k+1}). Equal to Algorithm 4
 * on constant-width (w = 1) cells. */
ORACLE_EXPORT double oracle_uniform_pairsum(const double *o, const double *l, int n, const struct oracle_params *p)
{
    if (n <= 0) return 0.0;
    double *pe = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *C = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    oracle_first_hit(o, n, pe);
    oracle_c_k(o, n, p->delta_occ, p->delta_emp, C);
    double H = (double)p->uniform_h;
    double I = 0.0;
    for (int j = p->e0_mode ? 0 : 1; j <= n; ++j) {
        double a = (j == 0) ? l[0] - 1.0 - H : l[j - 1] - H;
        double b = (j == 0) ? l[0] + H : l[j] + H;
        for (int k = 1; k <= n; ++k) {
            double lo = l[k - 1] > a ? l[k - 1] : a;
            double hi = l[k] < b ? l[k] : b;
            if (hi > lo) I += pe[j] * C[k - 1] * (hi - lo) / (b - a);
        }
    }
    free(pe);
    free(C);
    return I;
}

/* ------------------------------------------------------------------------------------------ */
/* 2D ray traversal (the paper lists "the cells the beam intersects", Section 2.2).            */
/* Fixed-point integer DDA: origin Q16 cell units, direction Q30; crossings decided by exact    */
/* int64 comparisons; a simultaneous x/y crossing is one diagonal step.                        */
/* ------------------------------------------------------------------------------------------ */

static int64_t floor_shift(int64_t v, int s)
{
    int64_t d = (int64_t)1 << s;
    return v >= 0 ? v / d : -((-v + d - 1) / d);
}

/* Direction of a beam: unit vector u (Q30) rotated by the pose's (cos, sin) (Q30), rounded
 * half up: d = floor((R u + 2^29) / 2^30). */
ORACLE_EXPORT void oracle_beam_dir_2d(const int32_t *pose, const int32_t *u, int32_t *d)
{
    int64_t c = pose[2], s = pose[3], ux = u[0], uy = u[1];
    d[0] = (int32_t)floor_shift(c * ux - s * uy + ((int64_t)1 << 29), 30);
    d[1] = (int32_t)floor_shift(s * ux + c * uy + ((int64_t)1 << 29), 30);
}

/* Cells visited by the segment from (ox, oy) along (dx, dy) with entry parameter < R.
 * cells[i] = cy*W + cx; l[i] = entry distance of cell i (l[0] = 0); l[n] = min(R, grid exit).
 * Returns n, or -1 if more than cap cells. Distance is the parameter lambda of
 * o + lambda * d / 2^30 (cell units). rfix = round(R * 2^16). */
static int trace_2d_end(int W, int H, int32_t ox, int32_t oy, int32_t dx, int32_t dy, int64_t rfix, int cap,
                        int32_t *cells, double *l, int *by_range);

ORACLE_EXPORT int oracle_trace_2d(int W, int H, int32_t ox, int32_t oy, int32_t dx, int32_t dy,
                                  int64_t rfix, int cap, int32_t *cells, double *l)
{
    int by_range;
    return trace_2d_end(W, H, ox, oy, dx, dy, rfix, cap, cells, l, &by_range);
}

/* The traversal itself; *by_range = 1 when the beam ended at the range limit R (inside the grid),
 * 0 when it left the grid first or crossed no cell. */
static int trace_2d_end(int W, int H, int32_t ox, int32_t oy, int32_t dx, int32_t dy, int64_t rfix, int cap,
                        int32_t *cells, double *l, int *by_range)
{
    *by_range = 0;
    if (dx == 0 && dy == 0) return 0;
    int64_t cx = floor_shift(ox, 16), cy = floor_shift(oy, 16);
    if (dx < 0 && (ox & 0xFFFF) == 0) cx -= 1; /* the cell entered by o + eps*d */
    if (dy < 0 && (oy & 0xFFFF) == 0) cy -= 1;
    if (cx < 0 || cx >= W || cy < 0 || cy >= H) return 0;
    int64_t adx = dx < 0 ? -(int64_t)dx : dx, ady = dy < 0 ? -(int64_t)dy : dy;
    int sx = dx > 0 ? 1 : -1, sy = dy > 0 ? 1 : -1;
    /* Q16 distance, along each axis, from the origin to the far side of the current cell */
    int64_t nx = dx > 0 ? (cx + 1) * 65536 - ox : ox - cx * 65536;
    int64_t ny = dy > 0 ? (cy + 1) * 65536 - oy : oy - cy * 65536;
    if (cap < 1) return -1;
    int n = 0;
    cells[n] = (int32_t)(cy * W + cx);
    l[n] = 0.0;
    n = 1;
    for (;;) {
        int stepx, stepy;
        if (dx == 0) { stepx = 0; stepy = 1; }
        else if (dy == 0) { stepx = 1; stepy = 0; }
        else {
            int64_t tx = nx * ady, ty = ny * adx; /* compare nx/adx with ny/ady */
            stepx = tx <= ty;
            stepy = ty <= tx;
        }
        int64_t num = stepx ? nx : ny, den = stepx ? adx : ady;
        if (!((num << 30) < rfix * den)) { /* next entry parameter >= R */
            l[n] = (double)rfix / 65536.0;
            *by_range = 1;
            break;
        }
        double lam = (double)num * 16384.0 / (double)den;
        if (stepx) { cx += sx; nx += 65536; }
        if (stepy) { cy += sy; ny += 65536; }
        if (cx < 0 || cx >= W || cy < 0 || cy >= H) {
            l[n] = lam;
            break;
        }
        if (n >= cap) return -1;
        cells[n] = (int32_t)(cy * W + cx);
        l[n] = lam;
        ++n;
    }
    return n;
}

static int64_t range_fix(double max_range) { return (int64_t)nearbyint(max_range * 65536.0); }

/* Batched 2D path: poses P x 4 (x, y in Q16; cos, sin of yaw in Q30), beam unit vectors
 * B x 2 (Q30), map W x H row-major o in [0, 1]; out[p*B + b] in nats. */
ORACLE_EXPORT void oracle_eval_2d(const float *map, int W, int H, const int32_t *poses, int P,
                                  const int32_t *dirs, int B, const struct oracle_params *p,
                                  double *out, int nthreads)
{
    int64_t rfix = range_fix(p->max_range);
    int cap = (int)(p->max_range * 1.5) + 4;
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1)
    for (long long i = 0; i < (long long)P * B; ++i) {
        int pi = (int)(i / B), bi = (int)(i % B);
        int32_t d[2];
        oracle_beam_dir_2d(poses + 4 * pi, dirs + 2 * bi, d);
        int32_t *cells = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
        double *l = (double *)malloc(sizeof(double) * (size_t)(cap + 1));
        double *o = (double *)malloc(sizeof(double) * (size_t)cap);
        int n = oracle_trace_2d(W, H, poses[4 * pi], poses[4 * pi + 1], d[0], d[1], rfix, cap, cells, l);
        if (n < 0) {
            out[i] = NAN;
        } else {
            for (int c = 0; c < n; ++c) o[c] = (double)map[cells[c]];
            out[i] = oracle_fsmi_beam(o, l, n, p);
        }
        free(cells);
        free(l);
        free(o);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Section 2.4: mutual information along discretised trajectories. The MI of a trajectory is the */
/* sum over its states of the scan MI (the sum over the state's beams, eq. mi_sum per beam);     */
/* a cell that contributed at an earlier state is marked and not used again. Within one state    */
/* the beams are summed as a scan, as in eq. (mi_sum) per beam.                                  */
/* ------------------------------------------------------------------------------------------ */

/* States of trajectory t are poses traj_off[t] .. traj_off[t+1]-1, in travel order.
 * beam_out[p*B + b], state_out[p] and traj_out[t] in nats. */
ORACLE_EXPORT void oracle_eval_trajectories_2d(const float *map, int W, int H, const int32_t *poses,
                                               const int32_t *traj_off, int T, const int32_t *dirs, int B,
                                               const struct oracle_params *p, double *beam_out,
                                               double *state_out, double *traj_out)
{
    int64_t rfix = range_fix(p->max_range);
    int cap = (int)(p->max_range * 1.5) + 4;
    unsigned char *counted = (unsigned char *)malloc((size_t)W * H);
    int32_t *cells = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *l = (double *)malloc(sizeof(double) * (size_t)(cap + 1));
    double *o = (double *)malloc(sizeof(double) * (size_t)cap);
    unsigned char *skip = (unsigned char *)malloc((size_t)cap);
    for (int t = 0; t < T; ++t) {
        memset(counted, 0, (size_t)W * H);
        double traj = 0.0;
        for (int pi = traj_off[t]; pi < traj_off[t + 1]; ++pi) {
            double scan = 0.0;
            /* the state's beams see only the marks of earlier states */
            for (int bi = 0; bi < B; ++bi) {
                int32_t d[2];
                oracle_beam_dir_2d(poses + 4 * pi, dirs + 2 * bi, d);
                int n = oracle_trace_2d(W, H, poses[4 * pi], poses[4 * pi + 1], d[0], d[1], rfix, cap, cells, l);
                double I = NAN;
                if (n >= 0) {
                    for (int c = 0; c < n; ++c) {
                        o[c] = (double)map[cells[c]];
                        skip[c] = counted[cells[c]] != 0;
                    }
                    I = oracle_fsmi_beam_skip(o, l, skip, n, p);
                }
                beam_out[(size_t)pi * B + bi] = I;
                scan += I;
            }
            /* then every cell the state's beams crossed is marked */
            for (int bi = 0; bi < B; ++bi) {
                int32_t d[2];
                oracle_beam_dir_2d(poses + 4 * pi, dirs + 2 * bi, d);
                int n = oracle_trace_2d(W, H, poses[4 * pi], poses[4 * pi + 1], d[0], d[1], rfix, cap, cells, l);
                for (int c = 0; c < n; ++c) counted[cells[c]] = 1;
            }
            state_out[pi] = scan;
            traj += scan;
        }
        traj_out[t] = traj;
    }
    free(counted);
    free(cells);
    free(l);
    free(o);
    free(skip);
}

/* ------------------------------------------------------------------------------------------ */
/* Eq. (bayesian_filter) with the inverse sensor model of eq. (inverse_sensing): for a beam that */
/* measured range z, the cell where z falls is updated by delta_occ and every cell the beam     */
/* crossed before it by delta_emp (odds multiplied); a beam with z >= max_range returned        */
/* nothing and updates every cell up to max_range by delta_emp. Beams are applied one after the */
/* other in (pose, beam) order, each as r <- r * delta, i.e. o <- o delta / (1 + o (delta-1)).  */
/* ------------------------------------------------------------------------------------------ */

static double odds_update(double o, double delta) { return o * delta / (1.0 + o * (delta - 1.0)); }

ORACLE_EXPORT void oracle_update_map_2d(double *map, int W, int H, const int32_t *poses, int P, const int32_t *dirs,
                                        int B, const float *ranges, const struct oracle_params *p)
{
    int64_t rmax = range_fix(p->max_range);
    int cap = (int)(p->max_range * 1.5) + 4;
    int32_t *cells = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    double *l = (double *)malloc(sizeof(double) * (size_t)(cap + 1));
    for (int pi = 0; pi < P; ++pi) {
        for (int bi = 0; bi < B; ++bi) {
            double z = (double)ranges[(size_t)pi * B + bi];
            if (!(z > 0.0)) continue; /* no measurement */
            int64_t rfix = rmax;
            int ret = 0; /* the beam returned at z < max_range */
            if (z < (double)rmax / 65536.0) {
                int64_t rz = range_fix(z);
                if (rz < rmax) {
                    rfix = rz;
                    ret = 1;
                }
            }
            int32_t d[2];
            oracle_beam_dir_2d(poses + 4 * pi, dirs + 2 * bi, d);
            int by_range;
            int n = trace_2d_end(W, H, poses[4 * pi], poses[4 * pi + 1], d[0], d[1], rfix, cap, cells, l, &by_range);
            for (int c = 0; c < n; ++c) {
                int occ = ret && by_range && c == n - 1;
                double *m = &map[cells[c]];
                if (*m > 0.0 && *m < 1.0) *m = odds_update(*m, occ ? p->delta_occ : p->delta_emp);
            }
        }
    }
    free(cells);
    free(l);
}

/* Batched explicit beams in CSR form: beam b has cells off[b]..off[b+1]-1 with occupancies o[]
 * and entry distances l[]; its end distance is lend[b]. */
ORACLE_EXPORT void oracle_eval_beams(const int *off, const float *o, const float *l, const float *lend,
                                     int nbeams, const struct oracle_params *p, double *out, int nthreads)
{
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1)
    for (int b = 0; b < nbeams; ++b) {
        int n = off[b + 1] - off[b];
        double *od = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        double *ld = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        for (int c = 0; c < n; ++c) {
            od[c] = (double)o[off[b] + c];
            ld[c] = (double)l[off[b] + c];
        }
        ld[n] = (double)lend[b];
        out[b] = oracle_fsmi_beam(od, ld, n, p);
        free(od);
        free(ld);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Section 4: 3D rays on equal virtual cells, run-length encoding                               */
/* ------------------------------------------------------------------------------------------ */

/* Ray direction: d_i = floor((sum_j R_ij u_j + 2^29) / 2^30); pose = x, y, z (Q16), R (Q30, row
 * major). Virtual cell i (0-based) is the voxel containing o + (i + 1/2) d, i.e. floor of the Q31
 * position (o << 15) + (2i + 1) d. Sampling stops at the first sample outside the grid.
 * Returns the number of samples written (<= nsamp). */
ORACLE_EXPORT int oracle_sample_3d(const float *vox, int X, int Y, int Z, const int32_t *pose,
                                   const int32_t *u, int nsamp, float *samples)
{
    int64_t d[3];
    for (int r = 0; r < 3; ++r) {
        int64_t acc = 0;
        for (int c = 0; c < 3; ++c) acc += (int64_t)pose[3 + 3 * r + c] * (int64_t)u[c];
        d[r] = floor_shift(acc + ((int64_t)1 << 29), 30);
    }
    int n = 0;
    for (int i = 0; i < nsamp; ++i) {
        int64_t v[3];
        for (int a = 0; a < 3; ++a)
            v[a] = floor_shift(((int64_t)pose[a] << 15) + (int64_t)(2 * i + 1) * d[a], 31);
        if (v[0] < 0 || v[0] >= X || v[1] < 0 || v[1] >= Y || v[2] < 0 || v[2] >= Z) break;
        samples[n++] = vox[((int64_t)v[2] * Y + v[1]) * X + v[0]];
    }
    return n;
}

/* Run-length encoding of eq. (occup_rle): maximal spans of bit-identical values, split greedily
 * from the sensor into runs of at most cap cells. Returns the run count. */
ORACLE_EXPORT int oracle_rle_encode(const float *s, int n, int cap, float *run_o, int *run_len)
{
    int nr = 0;
    for (int i = 0; i < n; ++i) {
        uint32_t a, b = 0;
        memcpy(&a, &s[i], 4);
        if (nr > 0) memcpy(&b, &run_o[nr - 1], 4);
        if (nr > 0 && a == b && run_len[nr - 1] < cap) {
            run_len[nr - 1] += 1;
        } else {
            run_o[nr] = s[i];
            run_len[nr] = 1;
            ++nr;
        }
    }
    return nr;
}

/* Noise kernel between virtual cells at index distance d (before normalisation):
 *  OG_PDF: exp(-d^2 / (2 sigma'^2)) (Theorem 3's G, normalised by 1/(sqrt(2 pi) sigma'));
 *  OG_ERF: Phi((d + 1/2)/sigma') - Phi((d - 1/2)/sigma') (Gaussian mass of the unit cell);
 *  box (uniform): 1[|d| <= H] (Theorem 6, normalised by 1/(2H+1)).
 * trunc >= 0 zeroes |d| > trunc (the strict band reading of Approx-FSMI-RLE). */
struct rle_kernel {
    int kind; /* 0 PDF, 1 ERF, 2 box */
    double sigma;
    int H;
    int trunc;
};

static double kern(const struct rle_kernel *K, int d)
{
    if (K->trunc >= 0 && abs(d) > K->trunc) return 0.0;
    if (K->kind == 2) return abs(d) <= K->H ? 1.0 : 0.0;
    if (K->kind == 1) return Phi((d + 0.5) / K->sigma) - Phi((d - 0.5) / K->sigma);
    return exp(-(double)d * (double)d / (2.0 * K->sigma * K->sigma));
}

static double kern_norm(const struct rle_kernel *K)
{
    if (K->kind == 2) return 1.0 / (2.0 * K->H + 1.0);
    if (K->kind == 1) return 1.0;
    return 1.0 / (sqrt(2.0 * M_PI) * K->sigma);
}

/* A[x, Lu, Lv, t] and B[x, Lu, Lv, t] of Theorem 3, summed from their definitions. */
static double rle_A(const struct rle_kernel *K, double x, int Lu, int Lv, int t)
{
    double s = 0.0;
    for (int j = 0; j < Lu; ++j)
        for (int k = 0; k < Lv; ++k) s += pow(x, j) * kern(K, j + t - k);
    return s;
}

static double rle_B(const struct rle_kernel *K, double x, int Lu, int Lv, int t)
{
    double s = 0.0;
    for (int j = 0; j < Lu; ++j)
        for (int k = 0; k < Lv; ++k) s += (double)k * pow(x, j) * kern(K, j + t - k);
    return s;
}

/* Exposed for the A/B t-shift identity tests: kind 0 PDF, 1 ERF, 2 box. */
ORACLE_EXPORT double oracle_rle_A(int kind, double sigma, int H, int trunc, double x, int Lu, int Lv, int t)
{
    struct rle_kernel K = {kind, sigma, H, trunc};
    return rle_A(&K, x, Lu, Lv, t);
}

ORACLE_EXPORT double oracle_rle_B(int kind, double sigma, int H, int trunc, double x, int Lu, int Lv, int t)
{
    struct rle_kernel K = {kind, sigma, H, trunc};
    return rle_B(&K, x, Lu, Lv, t);
}

/* FSMI-RLE (Theorem 3), Approx-FSMI-RLE (Theorem 5) and Uniform-FSMI-RLE (Theorem 6) on one
 * run-length-encoded ray of nr runs with occupancies ro[] and lengths rl[] (unit cells, w = 1). */
ORACLE_EXPORT double oracle_rle_beam(const float *ro, const int *rl, int nr, const struct oracle_params *p)
{
    if (nr <= 0) return 0.0;
    double *PE = (double *)malloc(sizeof(double) * (size_t)nr);
    double *DE = (double *)malloc(sizeof(double) * (size_t)nr);
    double *fo = (double *)malloc(sizeof(double) * (size_t)nr);
    double *fe = (double *)malloc(sizeof(double) * (size_t)nr);
    int *s = (int *)malloc(sizeof(int) * (size_t)nr);
    /* Algorithms for P_E(u) and D_E(v); s_u = sum_{i<u} L_i */
    PE[0] = 1.0;
    DE[0] = 0.0;
    s[0] = 0;
    for (int u = 0; u < nr; ++u) {
        double o = (double)ro[u];
        fo[u] = oracle_f_prob(p->delta_occ, o);
        fe[u] = oracle_f_prob(p->delta_emp, o);
        if (u + 1 < nr) {
            PE[u + 1] = PE[u] * pow(1.0 - o, rl[u]);
            DE[u + 1] = DE[u] + rl[u] * fe[u];
            s[u + 1] = s[u] + rl[u];
        }
    }
    struct rle_kernel K = {p->g_kernel == OG_ERF ? 1 : 0, p->sigma, p->uniform_h, -1};
    if (p->variant == OV_UNIFORM) K.kind = 2;
    int approx_b = (p->variant == OV_APPROX && p->approx_reading == 0);
    if (p->variant == OV_APPROX && p->approx_reading == 1) K.trunc = p->trunc_delta;
    double I = 0.0;
    if (!approx_b) {
        /* eq. (group_fsmi_rle_exact): all run pairs */
        for (int u = 0; u < nr; ++u) {
            double o = (double)ro[u], x = 1.0 - o;
            for (int v = 0; v < nr; ++v) {
                int t = s[u] - s[v];
                I += PE[u] * o * ((DE[v] + fo[v]) * rle_A(&K, x, rl[u], rl[v], t) + fe[v] * rle_B(&K, x, rl[u], rl[v], t));
            }
        }
    } else {
        /* Theorem 5 as printed: diagonal blocks untruncated (theta, gamma), off-diagonal pairs
         * restricted to the sub-blocks s', L' of eqs. (su')-(Lv'), shift t = s_u' - s_v'. */
        int Dl = p->trunc_delta;
        for (int u = 0; u < nr; ++u) {
            double o = (double)ro[u], x = 1.0 - o;
            int Lu = rl[u];
            I += PE[u] * o * ((DE[u] + fo[u]) * rle_A(&K, x, Lu, Lu, 0) + fe[u] * rle_B(&K, x, Lu, Lu, 0));
            for (int v = u + 1; v < nr; ++v) {
                if (!(s[v] < s[u] + Lu + Dl)) continue;
                int su2 = s[u] > s[v] - Dl ? s[u] : s[v] - Dl;
                int Lu2 = s[u] + Lu - su2;
                int sv2 = s[v];
                int Lv2 = rl[v] < s[u] + Lu + Dl - s[v] ? rl[v] : s[u] + Lu + Dl - s[v];
                int t = su2 - sv2;
                I += PE[u] * pow(x, su2 - s[u]) * o *
                     ((DE[v] + fo[v]) * rle_A(&K, x, Lu2, Lv2, t) + fe[v] * rle_B(&K, x, Lu2, Lv2, t));
            }
            for (int v = 0; v < u; ++v) {
                if (!(s[u] < s[v] + rl[v] + Dl)) continue;
                int su2 = s[u];
                int Lu2 = Lu < s[v] + rl[v] + Dl - s[u] ? Lu : s[v] + rl[v] + Dl - s[u];
                int sv2 = s[v] > s[u] - Dl ? s[v] : s[u] - Dl;
                int Lv2 = s[v] + rl[v] - sv2;
                int t = su2 - sv2;
                I += PE[u] * o *
                     ((DE[v] + (sv2 - s[v]) * fe[v] + fo[v]) * rle_A(&K, x, Lu2, Lv2, t) + fe[v] * rle_B(&K, x, Lu2, Lv2, t));
            }
        }
    }
    I *= kern_norm(&K);
    free(PE);
    free(DE);
    free(fo);
    free(fe);
    free(s);
    return I;
}

/* Batched RLE evaluation over a CSR of runs: ray r owns runs off[r]..off[r+1]-1. */
ORACLE_EXPORT void oracle_eval_rle(const int *off, const float *ro, const uint8_t *rl8, int nrays,
                                   const struct oracle_params *p, double *out, int nthreads)
{
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (int r = 0; r < nrays; ++r) {
        int nr = off[r + 1] - off[r];
        int *rl = (int *)malloc(sizeof(int) * (size_t)(nr + 1));
        for (int u = 0; u < nr; ++u) rl[u] = rl8[off[r] + u];
        out[r] = oracle_rle_beam(ro + off[r], rl, nr, p);
        free(rl);
    }
}

/* Batched 3D path: sample, encode and evaluate each of P x R rays; also returns the run count of
 * each ray. poses P x 12, ray unit vectors R x 3 (Q30). */
ORACLE_EXPORT void oracle_eval_3d(const float *vox, int X, int Y, int Z, const int32_t *poses, int P,
                                  const int32_t *dirs, int R, const struct oracle_params *p,
                                  double *out, int *nruns, int nthreads)
{
    int nsamp = (int)floor(p->max_range);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (long long i = 0; i < (long long)P * R; ++i) {
        int pi = (int)(i / R), ri = (int)(i % R);
        float *smp = (float *)malloc(sizeof(float) * (size_t)(nsamp + 1));
        float *ro = (float *)malloc(sizeof(float) * (size_t)(nsamp + 1));
        int *rl = (int *)malloc(sizeof(int) * (size_t)(nsamp + 1));
        int n = oracle_sample_3d(vox, X, Y, Z, poses + 12 * pi, dirs + 3 * ri, nsamp, smp);
        int nr = oracle_rle_encode(smp, n, p->run_cap, ro, rl);
        out[i] = oracle_rle_beam(ro, rl, nr, p);
        if (nruns) nruns[i] = nr;
        free(smp);
        free(ro);
        free(rl);
    }
}
