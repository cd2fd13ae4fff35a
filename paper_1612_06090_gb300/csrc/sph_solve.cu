// sph_solve.cu -- the pass loop around the density kernel: work items, the h update with
// its convergence test, the todo-list compaction and the scatter back to caller order.
//
// This is the lockless scheme of Sec. IV-A (Listing 3) on the GPU: every pass runs only
// over the todo list of unconverged particles; mark_for_recomputation becomes the h-update
// kernel plus a stable compaction that writes the next todo list; the error check that the
// listing hoists out of the loop is a device status word read once the pass loop is done.
#include <cfloat>
#include <cmath>

#include "sph_kernels.cuh"

namespace sph {

namespace {

constexpr int kThreads = 256;
constexpr double kGrowth = 1.2599210498948732;  // 2^(1/3), the bisection-free growth step

__device__ __forceinline__ int seg_of(uint64_t k, const KeyLayout &kl)
{
    return kl.seg_bits > 0 ? (int)(k >> (3 * kl.lmax)) : 0;
}

// Grouping level of a target: the finest octree level whose cell edge is at least
// h / 2^shift (so the targets of one work item lie within about h of each other).
// `big` marks targets whose cell plus h reaches half the periodic range; those form
// single-target work items so every staged offset is a minimum-image offset.
// (FP32 with margins that make `big` conservative; the level itself only steers efficiency)
// Expected neighbours within h from the local density of the dense cell table: the target's
// table cell, widened to coarser levels until it holds 8 particles.
__device__ __forceinline__ float expected_neighbours(uint64_t k, float h, const SegInfo &S,
                                                     const KeyLayout &kl, const int32_t *__restrict__ ctab)
{
    const int32_t *t = ctab + S.tab_off;
    const int lc = S.level_c;
    uint64_t m = (k & ((1ull << (3 * kl.lmax)) - 1ull)) >> (3 * (kl.lmax - lc));
    int l = lc;
    int cnt = t[m + 1] - t[m];
    while (cnt < 8 && l > 0) {
        l--;
        m >>= 3;
        const int sh = 3 * (lc - l);
        cnt = t[(m + 1) << sh] - t[m << sh];
    }
    float vol = 1.f;
    for (int d = 0; d < 3; d++) vol *= ldexpf((float)S.q[d], kl.coord_bits - l);
    return (float)cnt / vol * (4.18879020f * h * h * h);
}

// Smallest e with 2^e >= x, for a positive normal float x (exact, from the exponent bits).
__device__ __forceinline__ int ceil_log2f(float x)
{
    const int b = __float_as_int(x);
    return ((b >> 23) & 0xff) - 127 + ((b & 0x7fffff) != 0 ? 1 : 0);
}

// hmul >= 1 scales h for the single-target test only (the list radius when lists are recorded).
__device__ __forceinline__ void bucket_of(uint64_t k, float h, const SegInfo &S,
                                          const KeyLayout &kl, int shift, int &lvl,
                                          uint64_t &prefix, bool &big, const int32_t *ctab,
                                          float hmul = 1.0f)
{
    const int cb = kl.coord_bits;
    const float maxinv = (float)fmax(S.inv_q[0], fmax(S.inv_q[1], S.inv_q[2]));
    const float hu = fminf(ceilf(h * maxinv * (1.0f + 1.0f / 1048576.0f)) + 1.0f, 1e30f);
    const float edge = ldexpf(hu, -shift);
    // the finest level l <= lmax whose cell edge 2^(cb - l) is at least edge (0 if none)
    int l = cb - ceil_log2f(edge);
    l = l > kl.lmax ? kl.lmax : l < 0 ? 0 : l;
    // ctab given (first pass of batched groups): a target whose starting h holds few neighbours
    // groups two levels coarser, so neighbouring isolated targets share items instead of paying
    // an item each (the todo list is still complete there, so consecutive targets are neighbours)
    if (ctab && l >= 2 && expected_neighbours(k, h, S, kl, ctab) < 16.f) l -= 2;
    lvl = l;
    prefix = k >> (3 * (kl.lmax - l));
    const float hb = hmul > 1.0f ? fminf(ceilf(h * hmul * maxinv * (1.0f + 1.0f / 1048576.0f)) + 1.0f, 1e30f) : hu;
    big = S.periodic && ((float)(1ll << (cb - l)) + hb >= (float)(1ll << (cb - 1)));
}

__device__ void reset_state(DevState *ds, int64_t n, int max_iter)
{
    ds->todo_count = (int32_t)n;
    ds->todo_next = 0;
    ds->n_items = 0;
    ds->item_head = 0;
    ds->exceeded = 0;
    ds->pass = 0;
    ds->max_iter = max_iter;
    ds->loop_flag = n > 0 ? 1 : 0;
    ds->pass_count = 0;
    ds->pair_evals = 0ull;
    ds->pair_tests = 0ull;
    ds->list_evals = 0ull;
    for (int k = 0; k < kMaxPasses; k++) {
        ds->todo_per_pass[k] = 0;
        ds->pairs_per_pass[k] = 0ull;
    }
}

__global__ void k_solve_init(SolveArgs a, const double *__restrict__ h_in, int max_iter)
{
    const int64_t n = a.n;
    const double h_first = n > 0 ? h_in[0] : 0.0;
    int bad = 0, varies = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a.idx[p];
        const double hv = h_in[i];
        const SegInfo &S = a.segs[seg_of(a.key[p], a.kl)];
        if (!(hv > 0.0 && hv <= DBL_MAX) || (S.periodic && hv >= S.half_box)) bad |= kBadH;
        varies |= hv != h_first;
        a.h[p] = hv;
        a.h32[p] = (float)hv;
        a.hlo[p] = 0.0;
        a.hhi[p] = HUGE_VAL;
        a.e_h[p] = hv;
        a.todo[0][p] = (int32_t)p;
        if (a.lst) a.lst_n[p] = -1;  // lists belong to one solve
    }
    if (bad) atomicOr(&a.ds->status, bad);
    if (varies) atomicOr(&a.ds->h_varies, 1);  // cleared by the host before this kernel
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_state(a.ds, n, max_iter);
}

// Starting search radii of the kNN passes.  A caller radius <= 0 is replaced by an estimate:
// the particle's cell at the dense-table level, widened to coarser levels until it holds 32
// particles, gives a local number density, and the radius is the one whose ball would hold 1.25K
// particles at that density (capped below half the periodic box).  The radius only steers the
// passes; the selected h does not depend on it.
__global__ void k_knn_init(SolveArgs a, const double *__restrict__ h_in, int max_iter, int K)
{
    const int64_t n = a.n;
    int bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a.idx[p];
        const uint64_t key = a.key[p];
        const SegInfo &S = a.segs[seg_of(key, a.kl)];
        double hv = h_in[i];
        if (hv <= 0.0) {
            const int32_t *t = a.ctab + S.tab_off;
            const int lc = S.level_c;
            const uint64_t local = key & ((1ull << (3 * a.kl.lmax)) - 1ull);
            uint64_t m = local >> (3 * (a.kl.lmax - lc));
            int l = lc;
            int64_t cnt = (int64_t)t[m + 1] - t[m];
            while (cnt < 32 && l > 0) {
                l--;
                m >>= 3;
                const int sh = 3 * (lc - l);
                cnt = (int64_t)t[(m + 1) << sh] - t[m << sh];
            }
            double vol = 1.0;
            for (int d = 0; d < 3; d++) vol *= ldexp(S.q[d], a.kl.coord_bits - l);
            const double dens = (double)(cnt > 0 ? cnt : 1) / vol;
            hv = cbrt(3.0 * (1.25 * K) / (4.0 * 3.14159265358979323846 * dens));
            if (S.periodic) hv = fmin(hv, 0.999 * S.half_box);
        }
        if (!(hv > 0.0 && hv <= DBL_MAX) || (S.periodic && hv >= S.half_box)) bad |= kBadH;
        a.h[p] = hv;
        a.h32[p] = (float)hv;
        a.hlo[p] = 0.0;
        a.hhi[p] = HUGE_VAL;
        a.e_h[p] = hv;
        a.e_cnt[p] = -1;  // no selection yet
        a.todo[0][p] = (int32_t)p;
    }
    if (bad) atomicOr(&a.ds->status, bad);
    if (blockIdx.x == 0 && threadIdx.x == 0) reset_state(a.ds, n, max_iter);
}

// A pass evaluates pass_count entries: the whole todo list while the loop runs, none once it
// has converged or reached max_iter (so a pass queued after that is a no-op).
// The branch-free FP32 pair loop runs in the first pass of a solve from one common h: every
// target then has the same, usually generous, h, so nearly every step has a lane within h and
// skipping the body never pays; later passes (and batches) keep the body under its test.
__global__ void k_pass_begin(DevState *ds, int free_first)
{
    ds->item_head = 0;
    ds->todo_next = 0;
    const bool run = ds->todo_count > 0 && ds->pass < ds->max_iter;
    ds->pass_count = run ? ds->todo_count : 0;
    ds->dens_count = ds->pass_count;  // with cached lists, replaced by the entries that search
    ds->free_now = free_first && ds->pass == 0 && !ds->h_varies;
    if (run && ds->pass < kMaxPasses) ds->todo_per_pass[ds->pass] = ds->todo_count;
}

__global__ void k_pass_end(DevState *ds)
{
    if (ds->pass_count > 0) {
        ds->todo_count = ds->todo_next;
        ds->pass += 1;
    }
    ds->loop_flag = (ds->todo_count > 0 && ds->pass < ds->max_iter) ? 1 : 0;
}

// Device-side loop condition of the CUDA-graph pass loop.
__global__ void k_set_loop(cudaGraphConditionalHandle handle, const DevState *ds)
{
    cudaGraphSetConditional(handle, ds->loop_flag ? 1u : 0u);
}

// Work-item heads: a new item starts at every multiple of gmax (gmax_sparse once the todo list
// is sparse) and around single-target ("big") entries.  While the todo list is dense (at least 1/8 of the particles) consecutive
// targets stay together if they share an octree cell at the coarser of their two grouping
// levels and those levels differ by at most one; once it is sparse they must have the same
// level and share the cell at it (long runs of far-apart targets would otherwise stretch an
// item's query box).  The segment is part of every key, so items never cross segments.
// The item's query box uses the targets' actual bounds, so the rule only steers efficiency.
__global__ void k_item_flags(SolveArgs a, const int32_t *__restrict__ todo)
{
    const int T = a.ds->dens_count;
    const bool dense = 8 * (int64_t)T >= a.n;
    // the sparse-target rule: first pass of batched open groups (isolated halo particles)
    const int32_t *ctab0 = a.ds->pass == 0 && a.kl.seg_bits > 0 ? a.ctab : nullptr;
    const float hmul = a.lst ? a.list_margin * 1.001f : 1.0f;
    const int lane = threadIdx.x & 31;
    // lanes hold consecutive entries, so an entry's predecessor is the previous lane's entry
    // (lane 0 works its own out); the loop bound is the warp's first entry, so shuffles see the
    // whole warp
    const int shift = dense ? a.group_shift : a.sparse_shift;
    const int gm = dense ? a.gmax : a.gmax_sparse;
    for (int tb = blockIdx.x * blockDim.x + (threadIdx.x & ~31); tb < T; tb += gridDim.x * blockDim.x) {
        const int t = tb + lane;
        const bool have = t < T;
        uint64_t k = 0, pre = 0;
        int l = 0;
        bool big = false;
        if (have) {
            const int p = todo[t];
            k = a.key[p];
            bucket_of(k, a.h32[p], a.segs[seg_of(k, a.kl)], a.kl, shift, l, pre, big, ctab0, hmul);
        }
        uint64_t kp = __shfl_up_sync(kFull, k, 1), prep = __shfl_up_sync(kFull, pre, 1);
        int lp = __shfl_up_sync(kFull, l, 1);
        bool bigp = __shfl_up_sync(kFull, (int)big, 1) != 0;
        if (lane == 0 && have && t > 0) {
            const int pp = todo[t - 1];
            kp = a.key[pp];
            bucket_of(kp, a.h32[pp], a.segs[seg_of(kp, a.kl)], a.kl, shift, lp, prep, bigp, ctab0, hmul);
        }
        if (!have) continue;
        int head = (t % gm == 0) || big;
        if (!head) {
            if (dense) {
                const int m = lp < l ? lp : l;
                head = bigp || (l - lp > 1) || (lp - l > 1) ||
                       (k >> (3 * (a.kl.lmax - m))) != (kp >> (3 * (a.kl.lmax - m)));
            } else {
                head = bigp || lp != l || prep != pre;
            }
        }
        a.flags[t] = head;
    }
}

// Number of leading octree levels two keys share: -1 when they lie in different segments,
// kl.lmax when they are equal.  Two keys share the level-L cell iff the result is >= L.
__device__ __forceinline__ int common_levels(uint64_t a, uint64_t b, const KeyLayout &kl)
{
    const uint64_t x = a ^ b;
    if (x == 0ull) return kl.lmax;
    const int lz = __clzll((long long)x) - (64 - kl.key_bits);
    if (lz < kl.seg_bits) return -1;
    return (lz - kl.seg_bits) / 3;
}

constexpr int kCapTile = 256;  // todo entries per tile of the capped item rule (one per thread)
constexpr int kCapMax = 64;    // largest item cap
constexpr int kCapLevels = 6;  // levels examined below a target's grouping level

// Work-item heads with the item cap: an item is the coarsest octree cell, no coarser than the
// targets' grouping level and at most kCapLevels - 1 levels finer, whose run of consecutive
// todo targets has at most item_cap entries.  Runs nest (a cell's run is a union of its
// children's runs), so every target of such a run finds the same cell, and items are compact
// groups of nearby targets whatever the local density.  A run that fits is cut every gmax
// targets from its start (when item_cap > gmax); a run still longer than item_cap at the finest
// level examined is cut at every multiple of gmax in the todo list.  Both are properties of the
// run, so all its members apply the same cut and no item exceeds gmax.  Each tile of the todo list
// is staged with its keys in shared memory; a target finds its run at every examined level
// with one walk of at most item_cap entries in each direction.
__global__ void __launch_bounds__(kCapTile) k_item_flags_capped(SolveArgs a, const int32_t *__restrict__ todo)
{
    constexpr int kHalo = kCapMax + 2;
    __shared__ uint64_t sk[kCapTile + 2 * kHalo];
    __shared__ int sl[kCapTile + 1];  // entries base - 1 .. base + kCapTile - 1: level | big << 8
    const int T = a.ds->dens_count;
    const int cap = a.item_cap < kCapMax ? a.item_cap : kCapMax;
    const bool dense = 8 * (int64_t)T >= a.n;
    const int shift = dense ? a.group_shift : a.sparse_shift;
    const int gm = dense ? a.gmax : a.gmax_sparse;
    const int32_t *ctab0 = a.ds->pass == 0 && a.kl.seg_bits > 0 ? a.ctab : nullptr;
    const int ntiles = (T + kCapTile - 1) / kCapTile;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int base = tile * kCapTile;
        // sk[i] holds the key of entry base - kHalo + i (positions outside [0, T) are never read
        // as keys: the walks stop at 0 and at T)
        for (int i = threadIdx.x; i < kCapTile + 2 * kHalo; i += blockDim.x) {
            const int t = base - kHalo + i;
            sk[i] = (t >= 0 && t < T) ? a.key[todo[t]] : 0ull;
        }
        __syncthreads();
        // levels shared by entry u and its predecessor (-1: u starts a run at every level)
        auto dprev = [&](int u) -> int {
            if (u <= 0 || u >= T) return -1;
            const int i = u - base + kHalo;
            return common_levels(sk[i - 1], sk[i], a.kl);
        };
        // level of entry t, and the distance from the start of its item's run (-1: the run is
        // longer than item_cap)
        auto level_of = [&](int t, int &from_start) -> int {
            from_start = -1;
            const int p = todo[t];
            const uint64_t k = a.key[p];
            int lh;
            uint64_t pre;
            bool big;
            bucket_of(k, a.h32[p], a.segs[seg_of(k, a.kl)], a.kl, shift, lh, pre, big, ctab0,
                      a.lst ? a.list_margin * 1.001f : 1.0f);
            if (big) return lh | (1 << 8);
            const int nl = a.kl.lmax - lh + 1 < kCapLevels ? a.kl.lmax - lh + 1 : kCapLevels;
            // back[k]: entries from the start of the level-(lh + k) run to t inclusive;
            // fwd[k]: entries after t in that run; cap + 1 stands for "more than cap"
            int back[kCapLevels], fwd[kCapLevels];
#pragma unroll
            for (int q = 0; q < kCapLevels; q++) back[q] = fwd[q] = cap + 1;
            // walking outwards, finer levels meet their boundary first: levels kres.. are resolved
            int kres = nl;
            for (int j = 0; j <= cap && kres > 0; j++) {
                if (t - j < 0) break;
                const int d = dprev(t - j);
#pragma unroll
                for (int q = kCapLevels - 1; q >= 0; q--)
                    if (q < kres && d < lh + q) {
                        back[q] = j + 1;
                        kres = q;
                    }
            }
            kres = nl;
            for (int j = 1; j <= cap && kres > 0; j++) {
                const int d = dprev(t + j);  // -1 past the end of the list
#pragma unroll
                for (int q = kCapLevels - 1; q >= 0; q--)
                    if (q < kres && d < lh + q) {
                        fwd[q] = j - 1;
                        kres = q;
                    }
            }
            int q = 0;
            while (q < nl - 1 && back[q] + fwd[q] > cap) q++;
            if (back[q] + fwd[q] <= cap) from_start = back[q] - 1;
            return lh + q;
        };
        const int t = base + threadIdx.x;
        int from_start = -1;
        if (t < T) sl[threadIdx.x + 1] = level_of(t, from_start);
        if (threadIdx.x == 0 && t > 0 && t - 1 < T) {
            int dummy;
            sl[0] = level_of(t - 1, dummy);
        }
        __syncthreads();
        if (t < T) {
            const int me = sl[threadIdx.x + 1];
            int head = t == 0 || (me >> 8) != 0;
            if (!head) {
                const int prev = sl[threadIdx.x];
                const int lvl = me & 0xff;
                head = (prev >> 8) != 0 || (prev & 0xff) != lvl || dprev(t) < lvl;
                if (!head) head = from_start >= 0 ? from_start % gm == 0 : t % gm == 0;
            }
            a.flags[t] = head;
        }
        __syncthreads();
    }
}

// mark_for_recomputation: band test, bracket, Newton or fallback, box limit (FP64, IEEE
// roundings spelled out so no product is fused into an FMA).
__global__ void k_h_update(SolveArgs a, const int32_t *__restrict__ todo)
{
    const int T = a.ds->pass_count;
    int exceeded = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        const int p = todo[t];
        const SegInfo &S = a.segs[seg_of(a.key[p], a.kl)];
        const double h = a.h[p];  // the h this pass evaluated
        const bool f32 = a.precision != 0;
        const double nw = f32 ? (double)a.e_nw32[p] : a.e_nw[p];
        const double dnw = f32 ? (double)a.e_dnw32[p] : a.e_dnw[p];
        a.e_h[p] = h;
        int alive = 0;
        if (!(fabs(__dsub_rn(nw, S.nngb)) <= S.tol)) {
            double lo = a.hlo[p], hi = a.hhi[p];
            if (nw < S.nngb) lo = h;
            else hi = h;
            double hn = h;
            bool take = false;
            if (dnw > 0.0) {
                hn = __dsub_rn(h, __ddiv_rn(__dsub_rn(nw, S.nngb), dnw));
                take = hn > lo && hn < hi && hn >= __dmul_rn(0.5, h) && hn <= __dmul_rn(2.0, h);
            }
            if (!take) {
                const bool has_lo = lo > 0.0, has_hi = hi < HUGE_VAL;
                if (has_lo && has_hi) hn = __dmul_rn(0.5, __dadd_rn(lo, hi));
                else if (has_lo) hn = __dmul_rn(h, kGrowth);
                else hn = __ddiv_rn(h, kGrowth);
            }
            a.hlo[p] = lo;
            a.hhi[p] = hi;
            if (S.periodic && hn >= S.half_box) {
                exceeded++;
            } else {
                a.h[p] = hn;
                a.h32[p] = (float)hn;
                alive = 1;
            }
        }
        a.flags[t] = alive;
    }
    exceeded = warp_sum(exceeded);
    if ((threadIdx.x & 31) == 0 && exceeded) atomicAdd(&a.ds->exceeded, exceeded);
}

__global__ void k_scatter(SolveArgs a, double *__restrict__ h_out, double *__restrict__ rho_out,
                          int32_t *__restrict__ count_out, double *__restrict__ nw_out,
                          double *__restrict__ dnw_out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = a.idx[p];
        const bool f32 = a.precision != 0;
        if (h_out) h_out[i] = a.e_h[p];
        rho_out[i] = f32 ? (double)a.e_rho32[p] : a.e_rho[p];
        count_out[i] = a.e_cnt[p];
        if (nw_out) nw_out[i] = f32 ? (double)a.e_nw32[p] : a.e_nw[p];
        if (dnw_out) dnw_out[i] = f32 ? (double)a.e_dnw32[p] : a.e_dnw[p];
    }
}


// After the kNN passes: a selected particle already has its density (summed from the
// selection buffer); one that did not finish (pass or box limit) is evaluated at its last
// search radius by one density pass over just those particles.
__global__ void k_knn_finish(SolveArgs a)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < a.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double h = a.e_h[p];
        a.h[p] = h;
        a.h32[p] = (float)h;
        a.flags[p] = a.e_cnt[p] < 0 ? 1 : 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ds->pass = 0;
        a.ds->max_iter = 1;
        a.ds->pair_evals = 0ull;
        for (int k = 0; k < kMaxPasses; k++) a.ds->pairs_per_pass[k] = 0ull;
    }
}

// Neighbour export set-up: every caller index maps to no sample row, then each sample claims
// its target's entry (a claim that finds the entry taken, or an index outside [0, n), flags the
// sample list as bad).
__global__ void k_nb_clear(int32_t *__restrict__ nb_slot, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        nb_slot[i] = -1;
}

__global__ void k_nb_mark(int32_t *__restrict__ nb_slot, const int64_t *__restrict__ sample, int64_t n_sample,
                          int64_t n, int32_t *__restrict__ nb_cnt, DevState *ds)
{
    int bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_sample;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sample[k];
        nb_cnt[k] = 0;
        if (i < 0 || i >= n || atomicCAS(&nb_slot[i], -1, (int32_t)k) != -1) bad = 1;
    }
    if (bad) atomicOr(&ds->status, kBadSample);
}

int blocks_for(int64_t n, int cap)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace

// Work items of the dens_count entries of todo: head flags, then their positions.
cudaError_t launch_items(const SolveArgs &a, const int32_t *todo, cudaStream_t st)
{
    const int grid = blocks_for(a.n, a.grid_cap);
    if (a.item_cap > 0) k_item_flags_capped<<<grid, kCapTile, 0, st>>>(a, todo);
    else k_item_flags<<<grid, kThreads, 0, st>>>(a, todo);
    if (a.launches) *a.launches += 1;
    // item starts = positions of the head flags
    return compact_i32(a.flags, nullptr, a.items, nullptr, a.n, &a.ds->dens_count, &a.ds->n_items, a.scan_aux,
                       a.grid_cap, st, a.launches);
}

cudaError_t launch_solve_init(const SolveArgs &a, const double *h_in, int max_iter, cudaStream_t st)
{
    k_solve_init<<<blocks_for(a.n, a.grid_cap), kThreads, 0, st>>>(a, h_in, max_iter);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_pass(const SolveArgs &a, int cur, bool update, cudaStream_t st)
{
    const int32_t *todo = a.todo[cur];
    const int grid = blocks_for(a.n, a.grid_cap);
    k_pass_begin<<<1, 1, 0, st>>>(a.ds, a.free_first);
    if (a.launches) *a.launches += 1;
    cudaError_t e = cudaSuccess;
    if (a.dens_ev[0]) cudaEventRecord(a.dens_ev[0], st);
    // with cached lists: the targets whose list still covers their h are evaluated from it, the
    // others (flags) go on to the neighbour search through todo_s
    const int32_t *stodo = todo;
    if (a.lst) {
        e = launch_list_eval(a, todo, st);
        if (e != cudaSuccess) return e;
        e = compact_i32(a.flags, todo, a.todo_s, nullptr, a.n, &a.ds->pass_count, &a.ds->dens_count,
                        a.scan_aux, a.grid_cap, st, a.launches);
        if (e != cudaSuccess) return e;
        stodo = a.todo_s;
    }
    e = launch_items(a, stodo, st);
    if (e != cudaSuccess) return e;
    e = launch_density(a, stodo, st);
    if (e != cudaSuccess) return e;
    if (a.dens_ev[1]) cudaEventRecord(a.dens_ev[1], st);
    if (!update) return cudaGetLastError();
    k_h_update<<<grid, kThreads, 0, st>>>(a, todo);
    if (a.launches) *a.launches += 1;
    e = compact_i32(a.flags, todo, a.todo[1 - cur], nullptr, a.n, &a.ds->pass_count, &a.ds->todo_next,
                    a.scan_aux, a.grid_cap, st, a.launches);
    if (e != cudaSuccess) return e;
    k_pass_end<<<1, 1, 0, st>>>(a.ds);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_interact_pass(const SolveArgs &a, const InteractArgs &ia, cudaStream_t st)
{
    k_pass_begin<<<1, 1, 0, st>>>(a.ds, 0);
    if (a.launches) *a.launches += 1;
    cudaError_t e = launch_items(a, a.todo[0], st);
    if (e != cudaSuccess) return e;
    if (a.dens_ev[0]) cudaEventRecord(a.dens_ev[0], st);
    e = launch_interact(a, ia, a.todo[0], st);
    if (e != cudaSuccess) return e;
    if (a.dens_ev[1]) cudaEventRecord(a.dens_ev[1], st);
    return cudaGetLastError();
}

cudaError_t launch_set_loop(cudaGraphConditionalHandle handle, const DevState *ds, cudaStream_t st)
{
    k_set_loop<<<1, 1, 0, st>>>(handle, ds);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const SolveArgs &a, double *h_out, double *rho_out, int32_t *count_out,
                           double *nw_out, double *dnw_out, cudaStream_t st)
{
    k_scatter<<<blocks_for(a.n, a.grid_cap), kThreads, 0, st>>>(a, h_out, rho_out, count_out, nw_out,
                                                                 dnw_out);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}


cudaError_t launch_knn_pass(const SolveArgs &a, int cur, int k, cudaStream_t st)
{
    const int32_t *todo = a.todo[cur];
    k_pass_begin<<<1, 1, 0, st>>>(a.ds, a.free_first);
    if (a.launches) *a.launches += 1;
    if (a.dens_ev[0]) cudaEventRecord(a.dens_ev[0], st);
    cudaError_t e = launch_knn(a, todo, k, st);
    if (e != cudaSuccess) return e;
    if (a.dens_ev[1]) cudaEventRecord(a.dens_ev[1], st);
    e = compact_i32(a.flags, todo, a.todo[1 - cur], nullptr, a.n, &a.ds->pass_count, &a.ds->todo_next,
                    a.scan_aux, a.grid_cap, st, a.launches);
    if (e != cudaSuccess) return e;
    k_pass_end<<<1, 1, 0, st>>>(a.ds);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_knn_init(const SolveArgs &a, const double *h_in, int max_iter, int k, cudaStream_t st)
{
    k_knn_init<<<blocks_for(a.n, a.grid_cap), kThreads, 0, st>>>(a, h_in, max_iter, k);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_nb_setup(const SolveArgs &a, int32_t *nb_slot, const int64_t *sample, int64_t n_sample,
                            int32_t *nb_cnt, cudaStream_t st)
{
    k_nb_clear<<<blocks_for(a.n, a.grid_cap), kThreads, 0, st>>>(nb_slot, a.n);
    k_nb_mark<<<blocks_for(n_sample, a.grid_cap), kThreads, 0, st>>>(nb_slot, sample, n_sample, a.n, nb_cnt, a.ds);
    if (a.launches) *a.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_knn_finish(const SolveArgs &a, cudaStream_t st)
{
    k_knn_finish<<<blocks_for(a.n, a.grid_cap), kThreads, 0, st>>>(a);
    if (a.launches) *a.launches += 1;
    // the particles without a selection become the todo list of one density pass
    cudaError_t e = compact_i32(a.flags, nullptr, a.todo[0], nullptr, a.n, nullptr, &a.ds->todo_count,
                                a.scan_aux, a.grid_cap, st, a.launches);
    if (e != cudaSuccess) return e;
    return launch_pass(a, 0, false, st);
}

}  // namespace sph
