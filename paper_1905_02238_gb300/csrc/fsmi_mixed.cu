// One persistent launch over a stream of candidate sets of both kinds: 2D sets (beams through the
// occupancy grid, Section 3) and 3D sets (rays through voxel submaps, run-length encoded, Section 4).
// The sets form one ordered list of work items (a 2D beam or a 3D ray each); warps take items in
// that order from the work queue, so each set finishes roughly in arrival order, and the kernel can
// record when every item completed (from which per-set latencies follow).
#include "eval2d.cuh"
#include "evalrle.cuh"

namespace fsmi {

namespace {

// range classes per kind, by their upper bound in cells (about a factor 1.25 apart)
constexpr int kMixClasses = 16;
constexpr int kMixBuckets = 2 * kMixClasses;  // 2D classes 0..15, 3D classes 16..31 (one per lane of the plan warp)
__host__ __device__ constexpr int mix_bound(int c)
{
    return c == 0 ? 16 : c == 1 ? 24 : c == 2 ? 32 : c == 3 ? 48 : c == 4 ? 64 : c == 5 ? 80 : c == 6 ? 96
         : c == 7 ? 128 : c == 8 ? 160 : c == 9 ? 192 : c == 10 ? 256 : c == 11 ? 320 : c == 12 ? 384
         : c == 13 ? 512 : c == 14 ? 768 : 1024;
}
static_assert(kMixBuckets <= 32, "the plan warp keeps one class per lane");
// which kinds a launch of k_eval_mixed takes: both (the single launch), or one class's kind, 3D with
// the evaluation path its variant uses (as fsmi_eval_3d compiles one kernel per path)
enum { kMixAny = 0, kMix2D = 1, kMix3DOther = 2, kMix3DThm5 = 3 };

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

// ---- range classes -----------------------------------------------------------------------------
//
// A single launch must size every warp's shared arrays for the longest beam or ray of the whole
// stream. When the caller's workspace holds a plan, a one-warp pre-pass sorts the sets, in stream
// order, into range classes (2D and 3D separately, ranges up to 16, 24, 32, 48, 64, 80, 96, 128,
// 160, 192, 256, 320, 384, 512, 768, 1024 cells), and each class runs as its own persistent launch
// of a kernel that holds only its kind's path, sized for its bound; classes follow one another in
// the stream. A set whose descriptor fails the plan's checks (kind, offsets, range, contiguous
// outputs) makes the plan invalid: the class launches then return at once and the single launch
// runs instead, with its per-item checks.

struct MixedPlan {
    int valid, pad;
    int nsb[kMixBuckets];          // sets per class
    long long count[kMixBuckets];  // items per class
    // then int list[kMixBuckets][nsets] (set indices in stream order) and
    // long long pref[kMixBuckets][nsets + 1] (first item of each listed set within its class)
};

__host__ __device__ inline size_t plan_list_bytes(int nsets) { return ((size_t)kMixBuckets * nsets * 4 + 7) & ~(size_t)7; }

__device__ __forceinline__ long long warp_incl_add_ll(long long v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// class of a set (2D: 0..15, 3D: 16..31) or -1 if its descriptor is not one a class launch takes
__device__ __forceinline__ int mixed_class(const fsmi_set &st, const MixedSrc &src, const DevParams &p2,
                                           const DevParams &p3)
{
    if (st.npose < 0 || st.ndir < 1 || st.pose_offset < 0 || st.dir_offset < 0) return -1;
    if (st.kind == FSMI_SET_2D) {
        if (!src.has2d || !(st.max_range > 0.0f && st.max_range <= p2.rmax)) return -1;
        if ((long long)st.pose_offset + st.npose > src.P2 || (long long)st.dir_offset + st.ndir > src.B2) return -1;
        int c = 0;
        while (c < kMixClasses - 1 && st.max_range > (float)mix_bound(c)) ++c;
        return c;
    }
    if (st.kind == FSMI_SET_3D) {
        if (!src.has3d || !(st.max_range >= 1.0f && st.max_range <= (float)p3.nmax)) return -1;
        if (st.volume < 0 || st.volume >= src.nvol) return -1;
        if ((long long)st.pose_offset + st.npose > src.P3 || (long long)st.dir_offset + st.ndir > src.R3) return -1;
        int c = 0;  // by the range itself: a class launch takes ranges up to its bound (and its nmax)
        while (c < kMixClasses - 1 && st.max_range > (float)mix_bound(c)) ++c;
        return kMixClasses + c;
    }
    return -1;
}

// One warp: the sets' classes, per class the listed sets in stream order with their first items.
__global__ void __launch_bounds__(32) k_mixed_plan(MixedSrc src, DevParams p2, DevParams p3, long long nitems,
                                                   unsigned char *plan_raw)
{
    const int lane = lane_id(), nsets = src.nsets;
    MixedPlan *pl = reinterpret_cast<MixedPlan *>(plan_raw);
    int *list = reinterpret_cast<int *>(plan_raw + sizeof(MixedPlan));
    long long *pref = reinterpret_cast<long long *>(plan_raw + sizeof(MixedPlan) + plan_list_bytes(nsets));
    int nsb = 0;          // lane b: sets of class b so far
    long long cnt = 0;    // lane b: items of class b so far
    long long total = 0;  // items of every set so far
    bool valid = true;
    for (int base = 0; base < nsets; base += 32) {
        const int si = base + lane;
        fsmi_set st{};
        int cls = -2;  // -2: no set on this lane
        long long n = 0;
        if (si < nsets) {
            st = src.sets[si];
            cls = mixed_class(st, src, p2, p3);
            n = cls >= 0 ? (long long)st.npose * st.ndir : 0;
        }
        const long long incl = warp_incl_add_ll(n);
        // outputs must be contiguous, in set order, inside [0, nitems)
        const bool ok = cls == -2 || (cls >= 0 && st.out_offset == total + incl - n);
        valid = valid && __all_sync(kFull, ok);
        total += __shfl_sync(kFull, incl, 31);
        for (int b = 0; b < kMixBuckets; ++b) {
            const bool in = cls == b;
            const unsigned mask = __ballot_sync(kFull, in);
            if (!mask) continue;
            const long long ib = warp_incl_add_ll(in ? n : 0);
            const int nb = __shfl_sync(kFull, nsb, b);
            const long long cb = __shfl_sync(kFull, cnt, b);
            if (in) {
                const int pos = nb + __popc(mask & ((1u << lane) - 1u));
                list[(size_t)b * nsets + pos] = si;
                pref[(size_t)b * (nsets + 1) + pos] = cb + ib - n;
            }
            const long long tb = __shfl_sync(kFull, ib, 31);
            if (lane == b) {
                nsb += __popc(mask);
                cnt += tb;
            }
        }
    }
    valid = valid && total == nitems;
    if (lane < kMixBuckets) {
        pl->nsb[lane] = nsb;
        pl->count[lane] = cnt;
        pref[(size_t)lane * (nsets + 1) + nsb] = cnt;
    }
    if (lane == 0) pl->valid = valid ? 1 : 0;
}

// A class launch's per-warp record of the set its items come from: class items [lo, hi) belong to
// it, class item lo is output item0, its poses and directions start at pose / dir with ndir
// directions per pose, and the last item taken (class item next - 1) was pose kp, direction kd.
// The plan checked every descriptor (index ranges, ranges within bounds, volume index), so a
// class launch reads them once per set rather than once per item.
struct ClassCache {
    long long lo, hi, item0, next;
    const int32_t *pose, *dir;
    const float *vox;  // 3D: the set's volume
    long long rfix;    // 2D: Q16 range
    float rend;        // 2D: the range as float
    int X, Y, Z;       // 3D: the volume's extent
    int nsamp;         // 3D: virtual cells per ray
    int ndir, kp, kd;
};
constexpr int kSetCacheFloats = 32;  // 128 bytes per warp, keeping the next warp's arrays 16-byte aligned
static_assert(sizeof(ClassCache) <= kSetCacheFloats * sizeof(float), "class cache slot");

// 64 registers (4 blocks of 8 warps): the 2D path needs no more, and residency bounds this kernel
template <int VAR, int KIND>
__global__ void __launch_bounds__(kMaxWarps * 32, 4)
    k_eval_mixed(MixedSrc src, DevParams p2, DevParams p3, const __grid_constant__ RleTable tbl, long long nitems,
                 int stride2, int stride3, float *out,
                 unsigned long long *times, int *status, unsigned long long *queue, int chunk,
                 const unsigned char *plan_raw, int bucket)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // with a plan: a class launch (bucket >= 0) takes its class's items and runs only if the plan is
    // valid; the single launch (bucket < 0) runs only if it is not
    long long nloc = nitems;
    if (plan_raw) {
        const MixedPlan *pl = reinterpret_cast<const MixedPlan *>(plan_raw);
        const bool valid = pl->valid != 0;
        if (bucket < 0 ? valid : !valid) return;
        if (bucket >= 0) nloc = pl->count[bucket];
    }
    if (nloc <= 0) return;  // a class without sets
    // block: the RLE kernel table of the 3D parameters; then each warp's arrays, used by either kind
    RleBlock rb;
    rb.ts = table_spec(p3);
    rb.tab = (float2 *)smem_raw;
    rb.gtab = (float *)(smem_raw + (size_t)(2 * rb.ts.K + 2) * sizeof(float2));
    if (src.has3d) load_table(rb.tab, rb.gtab, rb.ts.K, tbl);
    const int per_warp = max(warp_floats_2d(stride2), ray3d_warp_floats(p3));  // then the set cache
    float *base = (float *)(smem_raw + rle_table_bytes(rb.ts.K)) + (size_t)(threadIdx.x >> 5) * (per_warp + kSetCacheFloats);
    rb.base = base;
    if (times && threadIdx.x == 0) atomicMin(times, global_ns());
    const int lane = lane_id();
    if (KIND != kMixAny) {  // a class launch of a valid plan: one kind, descriptors checked by the plan
        ClassCache *cc = reinterpret_cast<ClassCache *>(base + per_warp);
        if (lane == 0) {
            cc->lo = 0;
            cc->hi = 0;
        }
        __syncwarp();
        for_each_item(nloc, queue, chunk, [&](long long li) {
            long long kp, kd;
            if (li < cc->lo || li >= cc->hi) {  // the listed set holding class item li: the last with pref <= li
                // (the plan's lists are read here, not held in registers across the items)
                const MixedPlan *pl = reinterpret_cast<const MixedPlan *>(plan_raw);
                const int nsb = pl->nsb[bucket];
                const int *blist = reinterpret_cast<const int *>(plan_raw + sizeof(MixedPlan)) + (size_t)bucket * src.nsets;
                const long long *bpref = reinterpret_cast<const long long *>(plan_raw + sizeof(MixedPlan) +
                                                                             plan_list_bytes(src.nsets)) +
                                         (size_t)bucket * (src.nsets + 1);
                int lo = 0, len = nsb + 1;
                while (len > 0) {
                    const int half = len >> 1;
                    if (bpref[lo + half] <= li) {
                        lo += half + 1;
                        len -= half + 1;
                    } else {
                        len = half;
                    }
                }
                const int idx = min(lo - 1, nsb - 1);  // >= 0: li >= pref[0] = 0
                const fsmi_set st = src.sets[blist[idx]];
                const long long k = li - bpref[idx];
                kp = k / st.ndir;
                kd = k - kp * st.ndir;
                __syncwarp();
                if (lane == 0) {
                    cc->lo = bpref[idx];
                    cc->hi = bpref[idx + 1];
                    cc->item0 = st.out_offset;
                    cc->ndir = st.ndir;
                    if (KIND == kMix2D) {
                        cc->pose = src.poses2 + 4 * (size_t)st.pose_offset;
                        cc->dir = src.dirs2 + 2 * (size_t)st.dir_offset;
                        cc->rfix = __double2ll_rn((double)st.max_range * 65536.0);
                        cc->rend = (float)((double)cc->rfix * (1.0 / 65536.0));
                    } else {
                        const fsmi_volume v = src.vols[st.volume];
                        cc->pose = src.poses3 + 12 * (size_t)st.pose_offset;
                        cc->dir = src.dirs3 + 3 * (size_t)st.dir_offset;
                        cc->vox = v.vox;
                        cc->X = v.X;
                        cc->Y = v.Y;
                        cc->Z = v.Z;
                        cc->nsamp = (int)st.max_range;
                    }
                }
                __syncwarp();
            } else if (li == cc->next) {  // the item after the last one: the next direction
                kp = cc->kp;
                kd = cc->kd + 1;
                if (kd == cc->ndir) {
                    kd = 0;
                    ++kp;
                }
            } else {
                const long long k = li - cc->lo;
                const int nd = cc->ndir;
                kp = k <= 0x7fffffffLL ? (long long)((unsigned)k / (unsigned)nd) : k / nd;
                kd = k - kp * nd;
            }
            const long long item = cc->item0 + (li - cc->lo);
            float I;
            int bad = 0;
            if (KIND == kMix2D) {
                float *sl, *sc, *sp, *sx;
                carve_2d(base, stride2, sl, sc, sp, sx);
                const int32_t *d = cc->dir + 2 * kd;
                const int n = beam_cells<false>(src.map, src.W, src.H, src.gains, cc->pose + 4 * kp, d[0], d[1], cc->rfix,
                                                cc->rend, p2.nmax, p2, 0, nullptr, sl, sc, sp, sx, status);
                if (n >= 0) {
                    I = beam_sum<VAR>(p2, n, sl, sc, sp, sx);
                } else {
                    I = __int_as_float(0x7fc00000);
                    bad = FSMI_STATUS_BEAM_OVERFLOW;
                }
            } else {
                int nr = 0;
                constexpr int kMode = KIND == kMix3DThm5 ? kRay3dThm5 : kRay3dOther;
                I = ray_mi_fused<kMode>(cc->vox, cc->X, cc->Y, cc->Z, cc->pose + 12 * kp, cc->dir + 3 * kd, cc->nsamp, p3,
                                        rb.tab, rb.gtab, rb.ts.K, base, &nr);
            }
            __syncwarp();
            if (lane == 0) {
                out[item] = I;
                if (bad) set_status(status, bad);
                if (times) times[1 + item] = global_ns();
                cc->next = li + 1;
                cc->kp = (int)kp;
                cc->kd = (int)kd;
            }
            __syncwarp();
        });
        return;
    }
    // the single launch: every item's descriptor checked before it is used
    for_each_item(nloc, queue, chunk, [&](long long item) {
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
            I = ray_mi_fused<kRay3dAny>(v.vox, v.X, v.Y, v.Z, src.poses3 + 12 * pi, src.dirs3 + 3 * di, (int)st.max_range,
                                        p3, rb.tab, rb.gtab, rb.ts.K, base, &nr);
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

template <int VAR, int KIND = kMixAny>
cudaError_t launch_mixed_variant(const MixedSrc &src, const DevParams &p2, const DevParams &p3, long long nitems,
                                 float *out, unsigned long long *times, int *status, unsigned long long *queue,
                                 cudaStream_t s, const unsigned char *plan = nullptr, int bucket = -1)
{
    // a 3D class runs under the RLE family's schedule, like fsmi_eval_3d; everything else the 2D one
    const Schedule &sc = current_schedule(KIND == kMix3DOther || KIND == kMix3DThm5 ? FSMI_KIND_RLE : FSMI_KIND_2D);
    const int stride2 = stride_2d(p2.nmax);
    const int stride3 = ((p3.nmax + 2 * p3.K + 4) + 3) & ~3;
    const size_t per_warp = ((size_t)max(warp_floats_2d(stride2), ray3d_warp_floats(p3)) + kSetCacheFloats) * sizeof(float);
    const size_t table = rle_table_bytes(table_spec(p3).K);
    const int wpb = fit_warps(sc.warps_per_block, per_warp, table);
    const size_t smem = table + (size_t)wpb * per_warp;
    auto kern = k_eval_mixed<VAR, KIND>;
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
    if (times && !plan) {  // start = min over blocks (with a plan, the caller resets it once)
        e = cudaMemsetAsync(times, 0xFF, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    RleTable tbl{};
    if (src.has3d) fill_rle_table(p3, tbl);
    kern<<<(unsigned)grid, wpb * 32, smem, s>>>(src, p2, p3, tbl, nitems, stride2, stride3, out, times, status, queue,
                                                sc.queue_chunk > 0 ? sc.queue_chunk : 1, plan, bucket);
    return cudaGetLastError();
}

// The call with a plan: the pre-pass, one launch per range class that can hold sets (each sized
// for its class's bound), then the single launch, which returns at once unless the plan failed.
template <int VAR>
cudaError_t launch_mixed_planned(const MixedSrc &src, const DevParams &d2, const DevParams &d3, long long nitems,
                                 float *out, unsigned long long *times, int *status, unsigned long long *queue,
                                 unsigned char *plan, cudaStream_t s)
{
    k_mixed_plan<<<1, 32, 0, s>>>(src, d2, d3, nitems, plan);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (times) {
        e = cudaMemsetAsync(times, 0xFF, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    DevParams n2{}, n3{};  // inert parameters for the kind a class launch does not run
    n2.variant = FSMI_EXACT;
    n2.nmax = 1;
    n3.variant = FSMI_UNIFORM;
    n3.nmax = 1;
    n3.K = 0;
    n3.cell_runlen = 1;
    for (int c = 0; c < kMixClasses; ++c) {
        const float lo = c == 0 ? 0.0f : (float)mix_bound(c - 1);
        if (src.has2d && lo < d2.rmax) {
            DevParams p = d2;
            const double rb = fmin((double)mix_bound(c), (double)d2.rmax);
            p.nmax = (int)(rb * 1.41421357) + 3;  // as make_params: every beam of the class fits
            MixedSrc sc2 = src;
            sc2.has3d = false;
            e = launch_mixed_variant<VAR, kMix2D>(sc2, p, n3, nitems, out, times, status, queue, s, plan, c);
            if (e != cudaSuccess) return e;
        }
        if (src.has3d && lo < (float)d3.nmax) {
            DevParams p = d3;
            p.nmax = min(mix_bound(c), d3.nmax);
            MixedSrc sc3 = src;
            sc3.has2d = false;
            e = thm5_of(p) ? launch_mixed_variant<VAR, kMix3DThm5>(sc3, n2, p, nitems, out, times, status, queue, s,
                                                                  plan, kMixClasses + c)
                           : launch_mixed_variant<VAR, kMix3DOther>(sc3, n2, p, nitems, out, times, status, queue, s,
                                                                   plan, kMixClasses + c);
            if (e != cudaSuccess) return e;
        }
    }
    return launch_mixed_variant<VAR>(src, d2, d3, nitems, out, times, status, queue, s, plan, -1);
}

}  // namespace

cudaError_t launch_eval_mixed(const float *map, int W, int H, const float4 *gains, const int32_t *poses2, int P2,
                              const int32_t *dirs2, int B2, const DevParams *p2, const fsmi_volume *vols, int nvol,
                              const int32_t *poses3, int P3, const int32_t *dirs3, int R3, const DevParams *p3,
                              const fsmi_set *sets, int nsets, long long nitems, float *out, unsigned long long *times,
                              int *status, unsigned long long *queue, unsigned char *plan, cudaStream_t s)
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
    if (plan) {
        switch (d2.variant) {
            case FSMI_EXACT:
                if (d2.flags & FSMI_FLAG_FULL_SWEEP)
                    return launch_mixed_planned<kExactFullSweep>(src, d2, d3, nitems, out, times, status, queue, plan, s);
                return launch_mixed_planned<FSMI_EXACT>(src, d2, d3, nitems, out, times, status, queue, plan, s);
            case FSMI_APPROX:
                return launch_mixed_planned<FSMI_APPROX>(src, d2, d3, nitems, out, times, status, queue, plan, s);
            default: return launch_mixed_planned<FSMI_UNIFORM>(src, d2, d3, nitems, out, times, status, queue, plan, s);
        }
    }
    switch (d2.variant) {
        case FSMI_EXACT:
            if (d2.flags & FSMI_FLAG_FULL_SWEEP)
                return launch_mixed_variant<kExactFullSweep>(src, d2, d3, nitems, out, times, status, queue, s);
            return launch_mixed_variant<FSMI_EXACT>(src, d2, d3, nitems, out, times, status, queue, s);
        case FSMI_APPROX: return launch_mixed_variant<FSMI_APPROX>(src, d2, d3, nitems, out, times, status, queue, s);
        default: return launch_mixed_variant<FSMI_UNIFORM>(src, d2, d3, nitems, out, times, status, queue, s);
    }
}

template <int VAR>
static cudaError_t prepare_mixed_var()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_eval_mixed<VAR, kMixAny>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_mixed<VAR, kMix2D>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_mixed<VAR, kMix3DOther>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_eval_mixed<VAR, kMix3DThm5>);
    return e;
}

size_t mixed_plan_bytes(int nsets)
{
    return sizeof(MixedPlan) + plan_list_bytes(nsets) + (size_t)kMixBuckets * (nsets + 1) * sizeof(long long);
}

cudaError_t prepare_mixed()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_mixed_plan);
    if (e == cudaSuccess) e = prepare_mixed_var<FSMI_EXACT>();
    if (e == cudaSuccess) e = prepare_mixed_var<kExactFullSweep>();
    if (e == cudaSuccess) e = prepare_mixed_var<FSMI_APPROX>();
    if (e == cudaSuccess) e = prepare_mixed_var<FSMI_UNIFORM>();
    return e;
}

}  // namespace fsmi
