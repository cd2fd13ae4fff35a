// sph_items.cuh -- work-item geometry shared by the density pass and the kNN pass: the query
// box of a group of targets in 32-bit fixed point, the octree cells that meet it, and their
// particle ranges (dense cell table above its level, binary search on the sorted keys below).
#pragma once
#include <climits>

#include "sph_common.cuh"

namespace sph {

namespace {

constexpr int kMaxCells = 64;  // cells per item (4 per dimension)

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
    int qlo[3];       // the same bounds clamped to int32 (whole range for full dimensions),
    int qhi[3];       // which is all the per-candidate test needs
    int bmin[3];      // bounding box of the item's targets relative to X0
    int bmax[3];
    float hmax;       // largest h of the item's targets
    int full[3];      // periodic dimension covered entirely
    int level;        // enumeration level
    uint32_t c_lo[3]; // first cell per dimension
    int nc[3];        // cells per dimension
    int64_t cstart[3];  // start of the first cell relative to X0 (fixed point; non-full dims)
};

// All item geometry is bounds for culling, so it is computed in FP32 with margins that
// only ever enlarge it (FP64 arithmetic runs at a small fraction of the FP32 rate here).
__device__ __forceinline__ void item_setup(const SegInfo &S, const KeyLayout &kl, int cell_div,
                                           bool active, const uint4 &P, float hf, ItemGeom &G,
                                           int rel[3])
{
    const uint32_t pc[3] = {P.x, P.y, P.z};
    // h > 0, so the order of the float bit patterns is the order of the values
    const float hmax = __int_as_float(__reduce_max_sync(kFull, active ? __float_as_int(hf) : 0));
    const int cb = kl.coord_bits;
    const int64_t range = 1ll << cb;
    int64_t E = 0;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        G.X0[d] = __shfl_sync(kFull, pc[d], 0);
        rel[d] = (int32_t)(pc[d] - G.X0[d]);
        const int bmin = __reduce_min_sync(kFull, active ? rel[d] : INT_MAX);
        const int bmax = __reduce_max_sync(kFull, active ? rel[d] : INT_MIN);
        G.bmin[d] = bmin;
        G.bmax[d] = bmax;
        const int64_t H =
            (int64_t)fminf(ceilf(hmax * (float)S.inv_q[d] * (1.0f + 1.0f / 1048576.0f)) + 2.0f, 4.0e18f);
        G.lo[d] = (int64_t)bmin - H;
        G.hi[d] = (int64_t)bmax + H;
        // A periodic dimension whose query spans half the range or more is taken whole
        // (each cell once); below that the cells it meets are counted modulo 2^level.
        G.full[d] = S.periodic && (G.hi[d] - G.lo[d] + 1 >= range / 2);
        const int64_t ext = G.full[d] ? range : G.hi[d] - G.lo[d] + 1;
        E = ext > E ? ext : E;
        G.qlo[d] = G.full[d] ? INT_MIN : (int)(G.lo[d] < INT_MIN ? (int64_t)INT_MIN : G.lo[d]);
        G.qhi[d] = G.full[d] ? INT_MAX : (int)(G.hi[d] > INT_MAX ? (int64_t)INT_MAX : G.hi[d]);
    }
    G.hmax = hmax;
    // cells of at least E / cell_div: at most cell_div + 1 cells per dimension meet the query
    int l = kl.lmax;
    while (l > 0 && cell_div * (1ll << (cb - l)) < E) l--;
    if (S.periodic && l == 0) l = 1;  // keep shifts below 32; the level-1 cells cover the box
    G.level = l;
    const int s = cb - l;
    const uint32_t cmask = (uint32_t)((1ull << l) - 1);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (G.full[d]) {
            G.c_lo[d] = 0;
            G.nc[d] = 1 << l;
            G.cstart[d] = 0;
        } else if (S.periodic) {
            const uint32_t alo = G.X0[d] + (uint32_t)G.lo[d];
            const uint32_t ahi = G.X0[d] + (uint32_t)G.hi[d];
            G.c_lo[d] = alo >> s;
            G.nc[d] = (int)((((ahi >> s) - (alo >> s)) & cmask) + 1);
            G.cstart[d] = G.lo[d] - (int64_t)(alo & ((1u << s) - 1u));
        } else {
            int64_t alo = (int64_t)G.X0[d] + G.lo[d];
            int64_t ahi = (int64_t)G.X0[d] + G.hi[d];
            if (alo < 0) alo = 0;
            if (ahi > 2147483647ll) ahi = 2147483647ll;
            G.c_lo[d] = (uint32_t)(alo >> s);
            G.nc[d] = ahi >= alo ? (int)((ahi >> s) - (alo >> s) + 1) : 0;
            G.cstart[d] = ((alo >> s) << s) - (int64_t)G.X0[d];
        }
    }
}

// The staging geometry of an item in FP32 offset units.  The ball around the centre of the
// targets' box, of radius (half-diagonal + h_max), holds every candidate within h of some
// target; staging keeps the exact integer box test and adds this ball test (FP32, with a margin
// that covers the rounding of the offsets and the fixed-point quantisation).
// FP32 offsets are taken from the centre of the targets' box rather than the first target:
// the largest offset a near-boundary pair needs is then half the box plus h, which bounds the
// rounding of the FP32 distance test.  The origin moves to the centre (X0 + cen) once per item,
// with the query bounds and the targets' offsets `rel`; cc0 (the ball centre relative to the
// first target, for the cell culling) is found before the move, cc (relative to the new
// origin: 0 or half a unit per dimension) after it.
struct ItemBall {
    float cc0[3];
    float cc[3];
    float ball2;
};

__device__ __forceinline__ ItemBall item_recentre(ItemGeom &G, int rel[3], const float qf[3])
{
    ItemBall B;
#pragma unroll
    for (int d = 0; d < 3; d++) B.cc0[d] = 0.5f * ((float)G.bmin[d] + (float)G.bmax[d]) * qf[d];
    const float qm = fmaxf(qf[0], fmaxf(qf[1], qf[2]));
    float half2 = 0.f;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const float hx = 0.5f * (float)((int64_t)G.bmax[d] - (int64_t)G.bmin[d]) * qf[d];
        half2 = fmaf(hx, hx, half2);
        const int64_t sum = (int64_t)G.bmin[d] + (int64_t)G.bmax[d];
        const int64_t cen = sum >> 1;
        B.cc[d] = 0.5f * (float)(sum - 2 * cen) * qf[d];  // 0 or half a unit
        // the wrapped 32-bit differences from the new origin are exact: the true offset of any
        // candidate within h of a target of this item fits in 32 bits
        G.X0[d] += (uint32_t)cen;
        rel[d] = (int32_t)((uint32_t)rel[d] - (uint32_t)cen);
        if (!G.full[d]) {
            const int64_t lo = G.lo[d] - cen, hi = G.hi[d] - cen;
            G.qlo[d] = (int)(lo < INT_MIN ? (int64_t)INT_MIN : lo);
            G.qhi[d] = (int)(hi > INT_MAX ? (int64_t)INT_MAX : hi);
        }
    }
    const float Rm = (sqrtf(half2) + G.hmax) * (1.0f + 1e-5f) + 8.0f * qm;
    B.ball2 = Rm * Rm;
    return B;
}

// Ranges of the item's cells; lane holds cells lane + 32 k, k < K.  A cell that lies
// entirely outside the staging ball (centre cc, squared radius ball2, both in the FP32 offset
// units of the item) can hold no candidate, so its range is left empty: no lookup, no loads.
// The test only drops cells whose nearest point is farther than the ball radius by a
// relative 1e-4, far above the rounding of the FP32 cell bounds (a few 1e-7 of the extent).
template <int K = 2>
__device__ __forceinline__ void item_ranges(const ItemGeom &G, int g, const SegInfo &S,
                                            const KeyLayout &kl, const int32_t *__restrict__ ctab,
                                            const uint64_t *__restrict__ key, int ncell,
                                            const float cc[3], float ball2, const float qf[3],
                                            long long r[K])
{
    const int lane = lane_id();
    const uint32_t cmask = (uint32_t)((1ull << G.level) - 1);
    // first cell's start and the cell size per dimension in FP32 offset units (warp-uniform)
    float c0f[3], csf[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        csf[d] = (float)(1ll << (kl.coord_bits - G.level)) * qf[d];
        c0f[d] = (float)G.cstart[d] * qf[d];
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
        const int c = lane + 32 * k;
        r[k] = 0;
        if (c < ncell) {
            const int ix = c % G.nc[0];
            const int iy = (c / G.nc[0]) % G.nc[1];
            const int iz = c / (G.nc[0] * G.nc[1]);
            const int id[3] = {ix, iy, iz};
            float dist2 = 0.f;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if (G.full[d]) continue;
                const float flo = fmaf((float)id[d], csf[d], c0f[d]), fhi = flo + csf[d];
                const float dd = fmaxf(fmaxf(flo - cc[d], cc[d] - fhi), 0.f);
                dist2 = fmaf(dd, dd, dist2);
            }
            if (dist2 > ball2 * 1.0001f) continue;
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
        in = in && rj[d] >= G.qlo[d] && rj[d] <= G.qhi[d];
    }
    return in;
}

__device__ __forceinline__ double min_image64(double dx, double L)
{
    const double half = __dmul_rn(0.5, L);
    if (dx > half) return __dsub_rn(dx, L);
    if (dx < -half) return __dadd_rn(dx, L);
    return dx;
}

}  // namespace

}  // namespace sph
