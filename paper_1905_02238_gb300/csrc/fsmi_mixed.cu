// One persistent launch over a stream of candidate sets of both kinds: 2D sets (beams through the
// occupancy grid, Section 3) and 3D sets (rays through voxel submaps, run-length encoded, Section 4).
// The sets form one ordered list of work items (a 2D beam or a 3D ray each); warps take items in
// that order from the work queue, so each set finishes roughly in arrival order, and the kernel can
// record when every item completed (from which per-set latencies follow).
#include "eval2d.cuh"
#include "evalrle.cuh"

namespace fsmi {

namespace {

// the set holding item i (sets sorted by out_offset), or -1
__device__ __forceinline__ int mixed_set_of(const fsmi_set *sets, int nsets, long long i)
{
    int lo = 0, len = nsets;
    while (len > 0) {
        const int half = len >> 1;
        if (__ldg(&sets[lo + half].out_offset) <= i) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo - 1;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

struct MixedSrc {
    // 2D
    const float *map;
    int W, H;
    const float4 *gains;
    const int32_t *poses2;
    int P2;
    const int32_t *dirs2;
    int B2;
    bool has2d;
    // 3D
    const fsmi_volume *vols;
    int nvol;
    const int32_t *poses3;
    int P3;
    const int32_t *dirs3;
    int R3;
    bool has3d;
    // sets
    const fsmi_set *sets;
    int nsets;
};

// 64 registers (4 blocks of 8 warps): the 2D path needs no more, and residency bounds this kernel
template <int VAR>
__global__ void __launch_bounds__(kMaxWarps * 32, 4)
    k_eval_mixed(MixedSrc src, DevParams p2, DevParams p3, long long nitems, int stride2, int stride3, float *out,
                 unsigned long long *times, int *status, unsigned long long *queue, int chunk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // block: the RLE kernel table of the 3D parameters; then each warp's arrays, used by either kind
    RleBlock rb;
    rb.ts = table_spec(p3);
    rb.tab = (float2 *)smem_raw;
    double *gs = (double *)(smem_raw + (size_t)(2 * rb.ts.K + 2) * sizeof(float2));
    rb.gtab = (float *)(gs + rb.ts.K + 1);
    if (src.has3d) build_table(rb.tab, gs, rb.gtab, rb.ts.K, rb.ts.kind, rb.ts.sigma, rb.ts.H, rb.ts.band);
    const int per_warp = max(warp_floats_2d(stride2), ray3d_warp_floats(p3));
    float *base = (float *)(smem_raw + rle_table_bytes(rb.ts.K)) + (size_t)(threadIdx.x >> 5) * per_warp;
    rb.base = base;
    if (times && threadIdx.x == 0) atomicMin(times, global_ns());
    const int lane = lane_id();
    for_each_item(nitems, queue, chunk, [&](long long item) {
        const int si = mixed_set_of(src.sets, src.nsets, item);
        fsmi_set st{};
        bool ok = si >= 0;
        if (ok) st = src.sets[si];
        const long long k = item - st.out_offset;
        ok = ok && st.npose >= 0 && st.ndir > 0 && k >= 0 && k < (long long)st.npose * st.ndir && st.pose_offset >= 0 &&
             st.dir_offset >= 0;
        const long long pi = st.pose_offset + (ok ? k / st.ndir : 0), di = st.dir_offset + (ok ? k % st.ndir : 0);
        float I = __int_as_float(0x7fc00000);
        int bad = 0;
        if (ok && st.kind == FSMI_SET_2D && src.has2d && pi < src.P2 && di < src.B2 && st.max_range > 0.0f &&
            st.max_range <= p2.rmax) {
            const long long rfix = __double2ll_rn((double)st.max_range * 65536.0);
            const float rend = (float)((double)rfix * (1.0 / 65536.0));
            float *sl, *sc, *sp, *sx;
            carve_2d(base, stride2, sl, sc, sp, sx);
            const int n = beam_cells<false>(src.map, src.W, src.H, src.gains, src.poses2 + 4 * pi,
                                            src.dirs2[2 * di], src.dirs2[2 * di + 1], rfix, rend, p2.nmax, p2, 0,
                                            nullptr, sl, sc, sp, sx, status);
            if (n >= 0)
                I = beam_sum<VAR>(p2, n, sl, sc, sp, sx);
            else
                bad = FSMI_STATUS_BEAM_OVERFLOW;
        } else if (ok && st.kind == FSMI_SET_3D && src.has3d && pi < src.P3 && di < src.R3 && st.volume >= 0 &&
                   st.volume < src.nvol && st.max_range >= 1.0f && st.max_range <= (float)p3.nmax) {
            const fsmi_volume v = src.vols[st.volume];
            int nr = 0;
            I = ray_mi_fused<kRay3dAny>(v.vox, v.X, v.Y, v.Z, src.poses3 + 12 * pi, src.dirs3 + 3 * di, (int)st.max_range, p3,
                             rb.tab, rb.gtab, rb.ts.K, base, &nr);
        } else {
            bad = FSMI_STATUS_BAD_BEAM;  // a malformed descriptor is never used to index
        }
        if (lane == 0) {
            out[item] = I;
            if (bad) set_status(status, bad);
            if (times) times[1 + item] = global_ns();
        }
        __syncwarp();
    });
}

template <int VAR>
cudaError_t launch_mixed_variant(const MixedSrc &src, const DevParams &p2, const DevParams &p3, long long nitems,
                                 float *out, unsigned long long *times, int *status, unsigned long long *queue,
                                 cudaStream_t s)
{
    const Schedule &sc = current_schedule(FSMI_KIND_2D);
    const int stride2 = stride_2d(p2.nmax);
    const int stride3 = ((p3.nmax + 2 * p3.K + 4) + 3) & ~3;
    const size_t per_warp = (size_t)max(warp_floats_2d(stride2), ray3d_warp_floats(p3)) * sizeof(float);
    const size_t table = rle_table_bytes(table_spec(p3).K);
    const int wpb = fit_warps(sc.warps_per_block, per_warp, table);
    const size_t smem = table + (size_t)wpb * per_warp;
    auto kern = k_eval_mixed<VAR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (sc.blocks_per_sm > 0 && sc.blocks_per_sm < occ) occ = sc.blocks_per_sm;
    long long grid = (long long)sm_count() * occ;
    if (grid > (nitems + wpb - 1) / wpb) grid = (nitems + wpb - 1) / wpb;
    if (queue) {
        e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    if (times) {
        e = cudaMemsetAsync(times, 0xFF, sizeof(unsigned long long), s);  // start = min over blocks
        if (e != cudaSuccess) return e;
    }
    kern<<<(unsigned)grid, wpb * 32, smem, s>>>(src, p2, p3, nitems, stride2, stride3, out, times, status, queue,
                                                sc.queue_chunk > 0 ? sc.queue_chunk : 1);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_eval_mixed(const float *map, int W, int H, const float4 *gains, const int32_t *poses2, int P2,
                              const int32_t *dirs2, int B2, const DevParams *p2, const fsmi_volume *vols, int nvol,
                              const int32_t *poses3, int P3, const int32_t *dirs3, int R3, const DevParams *p3,
                              const fsmi_set *sets, int nsets, long long nitems, float *out, unsigned long long *times,
                              int *status, unsigned long long *queue, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    // a kind without parameters gets inert ones sized for nothing
    DevParams d2{}, d3{};
    d2.variant = FSMI_EXACT;
    d2.nmax = 1;
    d3.variant = FSMI_UNIFORM;
    d3.nmax = 1;
    d3.K = 0;
    d3.cell_runlen = 1;
    if (p2) d2 = *p2;
    if (p3) d3 = *p3;
    MixedSrc src{map, W, H, gains, poses2, P2, dirs2, B2, p2 != nullptr, vols, nvol, poses3, P3, dirs3, R3,
                 p3 != nullptr, sets, nsets};
    switch (d2.variant) {
        case FSMI_EXACT:
            if (d2.flags & FSMI_FLAG_FULL_SWEEP)
                return launch_mixed_variant<kExactFullSweep>(src, d2, d3, nitems, out, times, status, queue, s);
            return launch_mixed_variant<FSMI_EXACT>(src, d2, d3, nitems, out, times, status, queue, s);
        case FSMI_APPROX: return launch_mixed_variant<FSMI_APPROX>(src, d2, d3, nitems, out, times, status, queue, s);
        default: return launch_mixed_variant<FSMI_UNIFORM>(src, d2, d3, nitems, out, times, status, queue, s);
    }
}

cudaError_t prepare_mixed()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_eval_mixed<FSMI_EXACT>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_mixed<kExactFullSweep>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_mixed<FSMI_APPROX>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_mixed<FSMI_UNIFORM>);
    return e;
}

}  // namespace fsmi
