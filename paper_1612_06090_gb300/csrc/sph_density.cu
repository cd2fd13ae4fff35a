// sph_density.cu -- the density pass: neighbour search + kernel sums for every target on
// the todo list (Eq. 1 with the M4 kernel; the density loop of Listing 1).
//
// Work decomposition.  The todo list (sorted positions of unconverged particles, in Morton
// order) is cut into work items of up to 32 consecutive targets that share one octree cell
// at their grouping level.  A persistent grid of warps pops items from a device counter
// (the dynamic scheduling of Listing 3, without a lock).  Per item, the warp:
//   1. builds the item's query box Q = bounding box of the targets grown by h_max, in
//      32-bit fixed point relative to the first target;
//   2. picks the octree level whose cells are at least |Q|/3, so at most 4 x 4 x 4 cells
//      meet Q, and looks each cell's particle range up (dense table at or above the
//      table level, binary search on the sorted keys below it);
//   3. streams those ranges with coalesced 16-byte loads, keeps the particles inside Q
//      (ballot compaction) and stages them in shared memory as FP32 offsets from the
//      first target (formed exactly in integer arithmetic, then rounded once);
//   4. runs the pair loop with one target per lane over the staged candidates.
// FP32 path: r < h test, kernel weights and partial sums in FP32, every 32 candidates
// the partial sums enter compensated (Kahan) accumulators; the totals go to FP64.
// FP64 path: the staged FP32 offsets only pre-filter with a widened radius; every pair that
// passes is recomputed from the FP64 positions exactly as the FP64 reference formulae are
// written (IEEE roundings, no contraction), so neighbour sets and per-pair terms are the
// FP64 ones.
#include <climits>

#include "sph_kernels.cuh"

namespace sph {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kStage = 256;     // candidates staged per warp before a pair-loop flush
constexpr int kMaxCells = 64;   // cells per item (4 per dimension)
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Compensated accumulation (Kahan): s + (-c) tracks the exact running sum.
__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    float y = __fsub_rn(v, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

__device__ __forceinline__ int64_t lower_bound_key(const uint64_t *__restrict__ key, int64_t lo,
                                                   int64_t hi, uint64_t k)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (key[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Particle range [s, e) of the level-l cell with Morton code m in segment g.
__device__ __forceinline__ int2 cell_range(uint64_t m, int l, int g, const SegInfo &S,
                                           const KeyLayout &kl, const int32_t *__restrict__ ctab,
                                           const uint64_t *__restrict__ key)
{
    const int32_t *t = ctab + S.tab_off;
    const int lc = S.level_c;
    if (l <= lc) {
        const int sh = 3 * (lc - l);
        return make_int2(t[m << sh], t[(m + 1) << sh]);
    }
    const uint64_t anc = m >> (3 * (l - lc));
    int64_t lo = t[anc], hi = t[anc + 1];
    const uint64_t base = kl.seg_bits > 0 ? ((uint64_t)g << (3 * kl.lmax)) : 0ull;
    const int sh = 3 * (kl.lmax - l);
    const uint64_t k0 = base + (m << sh);
    const uint64_t k1 = base + ((m + 1) << sh);
    int64_t s = lower_bound_key(key, lo, hi, k0);
    int64_t e = lower_bound_key(key, s, hi, k1);
    return make_int2((int)s, (int)e);
}

// Warp-uniform geometry of one work item.
struct ItemGeom {
    uint32_t X0[3];   // fixed-point position of the first target
    int64_t lo[3];    // query box relative to X0, inclusive
    int64_t hi[3];
    int full[3];      // periodic dimension covered entirely
    int level;        // enumeration level
    uint32_t c_lo[3]; // first cell per dimension
    int nc[3];        // cells per dimension
};

__device__ __forceinline__ void item_setup(const SegInfo &S, const KeyLayout &kl, bool active,
                                           const uint4 &P, double hd, ItemGeom &G, int rel[3])
{
    const uint32_t pc[3] = {P.x, P.y, P.z};
    double hmax = active ? hd : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hmax = fmax(hmax, __shfl_xor_sync(kFull, hmax, o));
    const int cb = kl.coord_bits;
    const int64_t range = 1ll << cb;
    int64_t E = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        G.X0[d] = __shfl_sync(kFull, pc[d], 0);
        rel[d] = (int32_t)(pc[d] - G.X0[d]);
        const int bmin = __reduce_min_sync(kFull, active ? rel[d] : INT_MAX);
        const int bmax = __reduce_max_sync(kFull, active ? rel[d] : INT_MIN);
        const int64_t H = (int64_t)fmin(ceil(hmax * S.inv_q[d]) + 2.0, 4.0e18);
        G.lo[d] = (int64_t)bmin - H;
        G.hi[d] = (int64_t)bmax + H;
        // A periodic dimension whose query spans half the range or more is taken whole
        // (each cell once); below that the cells it meets are counted modulo 2^level.
        G.full[d] = S.periodic && (G.hi[d] - G.lo[d] + 1 >= range / 2);
        const int64_t ext = G.full[d] ? range : G.hi[d] - G.lo[d] + 1;
        E = ext > E ? ext : E;
    }
    int l = kl.lmax;
    while (l > 0 && 3 * (1ll << (cb - l)) < E) l--;
    if (S.periodic && l == 0) l = 1;  // keep shifts below 32; the level-1 cells cover the box
    G.level = l;
    const int s = cb - l;
    const uint32_t cmask = (uint32_t)((1ull << l) - 1);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (G.full[d]) {
            G.c_lo[d] = 0;
            G.nc[d] = 1 << l;
        } else if (S.periodic) {
            const uint32_t alo = G.X0[d] + (uint32_t)G.lo[d];
            const uint32_t ahi = G.X0[d] + (uint32_t)G.hi[d];
            G.c_lo[d] = alo >> s;
            G.nc[d] = (int)((((ahi >> s) - (alo >> s)) & cmask) + 1);
        } else {
            int64_t alo = (int64_t)G.X0[d] + G.lo[d];
            int64_t ahi = (int64_t)G.X0[d] + G.hi[d];
            if (alo < 0) alo = 0;
            if (ahi > 2147483647ll) ahi = 2147483647ll;
            G.c_lo[d] = (uint32_t)(alo >> s);
            G.nc[d] = ahi >= alo ? (int)((ahi >> s) - (alo >> s) + 1) : 0;
        }
    }
}

// Ranges of the item's cells; lane holds cells `lane` and `lane + 32`.
__device__ __forceinline__ void item_ranges(const ItemGeom &G, int g, const SegInfo &S,
                                            const KeyLayout &kl, const int32_t *__restrict__ ctab,
                                            const uint64_t *__restrict__ key, int ncell,
                                            long long r[2])
{
    const int lane = lane_id();
    const uint32_t cmask = (uint32_t)((1ull << G.level) - 1);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int c = lane + 32 * k;
        r[k] = 0;
        if (c < ncell) {
            const int ix = c % G.nc[0];
            const int iy = (c / G.nc[0]) % G.nc[1];
            const int iz = c / (G.nc[0] * G.nc[1]);
            const uint32_t cx = (G.c_lo[0] + ix) & cmask;
            const uint32_t cy = (G.c_lo[1] + iy) & cmask;
            const uint32_t cz = (G.c_lo[2] + iz) & cmask;
            const int2 se = cell_range(morton3(cx, cy, cz), G.level, g, S, kl, ctab, key);
            r[k] = (long long)(unsigned)se.x | ((long long)se.y << 32);
        }
    }
}

__device__ __forceinline__ bool in_query(const ItemGeom &G, const uint4 &Pj, int rj[3])
{
    const uint32_t pc[3] = {Pj.x, Pj.y, Pj.z};
    bool in = true;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        rj[d] = (int32_t)(pc[d] - G.X0[d]);
        in = in && (G.full[d] || ((int64_t)rj[d] >= G.lo[d] && (int64_t)rj[d] <= G.hi[d]));
    }
    return in;
}

struct Acc32 {
    float s_mw, c_mw, s_w, c_w, s_dw, c_dw;
    int count;
};

// FP32 pair loop: lanes are targets, candidates are broadcast from shared memory.
__device__ __forceinline__ void flush_f32(const float4 *__restrict__ stage, int cnt, float tx,
                                          float ty, float tz, float h2f, float hinv2, Acc32 &A)
{
    for (int j0 = 0; j0 < cnt; j0 += 32) {
        const int j1 = j0 + 32 < cnt ? j0 + 32 : cnt;
        float pmw = 0.f, pw = 0.f, pdw = 0.f;
        int pc = 0;
        for (int j = j0; j < j1; j++) {
            const float4 c = stage[j];
            const float dx = c.x - tx, dy = c.y - ty, dz = c.z - tz;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 < h2f) {
                // M4 as a B-spline: w = 2 (1-q)^3 - 8 max(0, 1/2-q)^3,
                // -q w' = 6 q ((1-q)^2 - 4 max(0, 1/2-q)^2)
                const float q = sqrt_approx(r2 * hinv2);
                const float a = 1.f - q;
                const float b = fmaxf(0.5f - q, 0.f);
                const float a2 = a * a, b2 = b * b;
                const float w = fmaf(2.f * a, a2, -8.f * b * b2);
                const float dw = 6.f * q * fmaf(-4.f, b2, a2);
                pmw = fmaf(c.w, w, pmw);
                pw += w;
                pdw += dw;
                pc++;
            }
        }
        kahan_add(A.s_mw, A.c_mw, pmw);
        kahan_add(A.s_w, A.c_w, pw);
        kahan_add(A.s_dw, A.c_dw, pdw);
        A.count += pc;
    }
}

// ---- FP64 pair terms, written as the FP64 reference writes them --------------------------
__device__ __forceinline__ double min_image64(double dx, double L)
{
    const double half = __dmul_rn(0.5, L);
    if (dx > half) return __dsub_rn(dx, L);
    if (dx < -half) return __dadd_rn(dx, L);
    return dx;
}

__device__ __forceinline__ double w64(double q)
{
    if (q <= 0.5) {
        const double t = __dsub_rn(__dmul_rn(6.0, q), 6.0);
        return __dadd_rn(1.0, __dmul_rn(__dmul_rn(q, q), t));
    }
    if (q < 1.0) {
        const double a = __dsub_rn(1.0, q);
        return __dmul_rn(2.0, __dmul_rn(__dmul_rn(a, a), a));
    }
    return 0.0;
}

__device__ __forceinline__ double mqdw64(double q)
{
    if (q <= 0.5) return __dmul_rn(__dmul_rn(q, q), __dsub_rn(12.0, __dmul_rn(18.0, q)));
    if (q < 1.0) {
        const double a = __dsub_rn(1.0, q);
        return __dmul_rn(__dmul_rn(6.0, q), __dmul_rn(a, a));
    }
    return 0.0;
}

struct Acc64 {
    double s_mw, s_w, s_dw;
    int count;
};

__device__ __forceinline__ void flush_f64(const float4 *__restrict__ stage,
                                          const int *__restrict__ sidx, int cnt, float tx, float ty,
                                          float tz, float h2loose, const double4_32a &ti, double h,
                                          double h2, const SegInfo &S,
                                          const double4_32a *__restrict__ pdbl, Acc64 &A)
{
    for (int j = 0; j < cnt; j++) {
        const float4 c = stage[j];
        const float dxf = c.x - tx, dyf = c.y - ty, dzf = c.z - tz;
        const float r2f = fmaf(dxf, dxf, fmaf(dyf, dyf, dzf * dzf));
        if (r2f < h2loose) {
            const double4_32a cj = pdbl[sidx[j]];
            double dx = __dsub_rn(cj.x, ti.x);
            double dy = __dsub_rn(cj.y, ti.y);
            double dz = __dsub_rn(cj.z, ti.z);
            if (S.periodic) {
                dx = min_image64(dx, S.box[0]);
                dy = min_image64(dy, S.box[1]);
                dz = min_image64(dz, S.box[2]);
            }
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz));
            if (r2 < h2) {
                const double q = __ddiv_rn(__dsqrt_rn(r2), h);
                const double w = w64(q);
                A.s_mw = __dadd_rn(A.s_mw, __dmul_rn(cj.w, w));
                A.s_w = __dadd_rn(A.s_w, w);
                A.s_dw = __dadd_rn(A.s_dw, mqdw64(q));
                A.count++;
            }
        }
    }
}

template <bool kF64>
__global__ void __launch_bounds__(kThreads, 2) k_density(SolveArgs a, const int32_t *__restrict__ todo)
{
    __shared__ float4 stage_all[kWarps][kStage];
    __shared__ int sidx_all[kF64 ? kWarps : 1][kF64 ? kStage : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *stage = stage_all[warp];
    int *sidx = sidx_all[kF64 ? warp : 0];
    const int n_items = a.ds->n_items;
    const int todo_count = a.ds->todo_count;
    unsigned long long pairs = 0;

    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&a.ds->item_head, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const int t0 = a.items[it];
        const int t1 = it + 1 < n_items ? a.items[it + 1] : todo_count;
        const bool active = lane < t1 - t0;
        const int p = todo[active ? t0 + lane : t0];
        const uint4 P = a.pfix[p];
        const double hd = a.h[p];
        const int g = a.kl.seg_bits > 0 ? (int)(a.key[p] >> (3 * a.kl.lmax)) : 0;
        const SegInfo &S = a.segs[g];

        ItemGeom G;
        int rel[3];
        item_setup(S, a.kl, active, P, hd, G, rel);
        const float qf[3] = {(float)S.q[0], (float)S.q[1], (float)S.q[2]};
        const float tx = (float)rel[0] * qf[0];
        const float ty = (float)rel[1] * qf[1];
        const float tz = (float)rel[2] * qf[2];
        const float hf = (float)hd;
        const float h2f = hf * hf;
        const float hinv2 = 1.0f / h2f;
        // FP64 path: widened radius for the pre-filter (rounding of the FP32 offsets and the
        // fixed-point quantisation both stay far inside the margin)
        const double qmax = fmax(S.q[0], fmax(S.q[1], S.q[2]));
        const float hl = (float)(hd * (1.0 + 1e-4) + 4.0 * qmax);
        const float h2loose = hl * hl;
        double4_32a ti = make_double4_32a(0, 0, 0, 0);
        if (kF64) ti = a.pdbl[p];

        const int ncell = G.nc[0] * G.nc[1] * G.nc[2];
        if (ncell > kMaxCells) {  // cannot happen by construction; report, never overrun
            if (lane == 0) atomicOr(&a.ds->status, 8);
            continue;
        }
        long long rr[2];
        item_ranges(G, g, S, a.kl, a.ctab, a.key, ncell, rr);

        Acc32 A32 = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
        Acc64 A64 = {0.0, 0.0, 0.0, 0};
        int cnt = 0;
        for (int c = 0; c < ncell; c++) {
            const long long rc = __shfl_sync(kFull, (c < 32) ? rr[0] : rr[1], c & 31);
            const int2 r = make_int2((int)(rc & 0xffffffffll), (int)(rc >> 32));
            for (int base = r.x; base < r.y; base += 32) {
                const int j = base + lane;
                int rj[3] = {0, 0, 0};
                uint4 Pj = make_uint4(0, 0, 0, 0);
                bool in = false;
                if (j < r.y) {
                    Pj = a.pfix[j];
                    in = in_query(G, Pj, rj);
                }
                const unsigned m = __ballot_sync(kFull, in);
                if (in) {
                    const int slot = cnt + __popc(m & lanemask_lt());
                    stage[slot] = make_float4((float)rj[0] * qf[0], (float)rj[1] * qf[1],
                                              (float)rj[2] * qf[2], __uint_as_float(Pj.w));
                    if (kF64) sidx[slot] = j;
                }
                cnt += __popc(m);
                if (cnt > kStage - 32) {
                    __syncwarp();
                    if (kF64) flush_f64(stage, sidx, cnt, tx, ty, tz, h2loose, ti, hd, hd * hd, S, a.pdbl, A64);
                    else flush_f32(stage, cnt, tx, ty, tz, h2f, hinv2, A32);
                    __syncwarp();
                    cnt = 0;
                }
            }
        }
        __syncwarp();
        if (cnt > 0) {
            if (kF64) flush_f64(stage, sidx, cnt, tx, ty, tz, h2loose, ti, hd, hd * hd, S, a.pdbl, A64);
            else flush_f32(stage, cnt, tx, ty, tz, h2f, hinv2, A32);
        }
        __syncwarp();

        if (active) {
            double smw, sw, sdw;
            int count;
            if (kF64) {
                smw = A64.s_mw;
                sw = A64.s_w;
                sdw = A64.s_dw;
                count = A64.count;
            } else {
                smw = (double)A32.s_mw - (double)A32.c_mw;
                sw = (double)A32.s_w - (double)A32.c_w;
                sdw = (double)A32.s_dw - (double)A32.c_dw;
                count = A32.count;
            }
            const double h = hd;
            a.e_h[p] = h;
            a.e_rho[p] = smw * (8.0 / (kPi * h * h * h));
            a.e_nw[p] = (32.0 / 3.0) * sw;
            a.e_dnw[p] = (32.0 / 3.0) * sdw / h;
            a.e_cnt[p] = count;
            pairs += (unsigned long long)count;
        }
    }
    pairs = warp_sum(pairs);
    if (lane == 0 && pairs) atomicAdd(&a.ds->pair_evals, pairs);
}

}  // namespace

int density_blocks_per_sm(int precision)
{
    int b = 0;
    if (precision == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_density<true>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_density<false>, kThreads, 0);
    return b > 0 ? b : 1;
}

cudaError_t launch_density(const SolveArgs &a, const int32_t *todo, cudaStream_t st)
{
    if (a.precision == 0) k_density<true><<<a.density_grid, kThreads, 0, st>>>(a, todo);
    else k_density<false><<<a.density_grid, kThreads, 0, st>>>(a, todo);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

}  // namespace sph
