// sph_sort.cu -- spatial ordering: fixed-point coordinates, Morton keys, LSD radix sort,
// gather into the sorted SoA and the dense per-segment cell tables.
//
// The paper's neighbour search walks a Barnes-Hut octree stored as a flat array (Sec. II-A);
// here the octree is implicit: particles sorted by Morton key make every octree cell a
// contiguous range, found in O(1) from a dense start table at one level per segment and by
// binary search on the keys below it.  The gather into a compact sorted SoA plays the role
// of the paper's AoS->SoA gather (Sec. IV-B).
#include <cfloat>
#include <climits>
#include <cmath>

#include "sph_common.cuh"
#include "sph_kernels.cuh"

namespace sph {

namespace {

constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kSortThreads = 256;     // 8 warps per block
constexpr int kTileKeys = 4096;       // keys per block tile in the radix passes
constexpr int kKeysPerThread = kTileKeys / kSortThreads;
constexpr int kWarpKeys = kTileKeys / (kSortThreads / 32);  // contiguous keys ranked by one warp
static_assert(kSortThreads == kRadixBins, "one thread per digit in the tile offsets");

// FP64 instructions issue at a small fraction of the FP32 rate on this GPU, so the key and
// gather kernels spend them only on the one multiply per coordinate that exact fixed point
// needs; rounding, wrapping and the input checks use a conversion and integer operations.

// Periodic fixed point: nearest multiple of q = L / 2^32 (ties to even), wrapped (L itself
// maps to 0).  The conversion saturates (negatives give 0), the wrap of 2^32 to 0 is the
// truncation to 32 bits, and a position outside [0, L) is flagged by the caller.
__device__ __forceinline__ uint32_t fix_periodic(double x, double inv_q)
{
    return (uint32_t)__double2ull_rn(x * inv_q);
}

// Open boundaries: nearest multiple of q above the origin, clamped to [0, 2^31).
__device__ __forceinline__ uint32_t fix_open(double x, double origin, double inv_q)
{
    const long long t = __double2ll_rn((x - origin) * inv_q);  // saturating conversion
    return (uint32_t)(t < 0 ? 0ll : t > 2147483647ll ? 2147483647ll : t);
}

// 0 <= x < L on the IEEE-754 bit patterns (L positive and finite; -0.0 counts as 0): a
// non-negative double orders like its bits, and NaN, infinities and negatives fail.
__device__ __forceinline__ bool in_range_bits(double x, long long l_bits)
{
    const long long b = __double_as_longlong(x);
    return (unsigned long long)b < (unsigned long long)l_bits || b == LLONG_MIN;
}

// 0 < m <= DBL_MAX on the bit pattern.
__device__ __forceinline__ bool positive_finite_bits(double m)
{
    return (unsigned long long)__double_as_longlong(m) - 1ull < 0x7fefffffffffffffull;
}

// |x| <= DBL_MAX on the bit pattern (not NaN, not infinite).
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) <= 0x7fefffffffffffffull;
}

// rec (nullable): the particle's 16-byte fixed-point record {X, Y, Z, FP32 mass}, written in
// caller order while the caller's arrays stream through, so the gather moves one record per
// particle instead of four scattered 8-byte reads (FP32 solves read nothing else).
__global__ void k_keys_periodic(int64_t n, const double *__restrict__ pos,
                                const double *__restrict__ mass, SegInfo seg, KeyLayout kl,
                                double box_x, double box_y, double box_z,
                                uint64_t *__restrict__ key, int32_t *__restrict__ idx,
                                DevState *ds, uint4 *__restrict__ rec)
{
    const int shift = kl.coord_bits - kl.lmax;
    const long long bx = __double_as_longlong(box_x), by = __double_as_longlong(box_y),
                    bz = __double_as_longlong(box_z);
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double x = pos[i], y = pos[n + i], z = pos[2 * n + i], m = mass[i];
        if (!(in_range_bits(x, bx) && in_range_bits(y, by) && in_range_bits(z, bz)))
            bad |= kBadPosition;
        if (!positive_finite_bits(m)) bad |= kBadMass;
        uint32_t X = fix_periodic(x, seg.inv_q[0]);
        uint32_t Y = fix_periodic(y, seg.inv_q[1]);
        uint32_t Z = fix_periodic(z, seg.inv_q[2]);
        key[i] = morton3(X >> shift, Y >> shift, Z >> shift);
        idx[i] = (int32_t)i;
        if (rec) rec[i] = make_uint4(X, Y, Z, __float_as_uint((float)m));
    }
    if (bad) atomicOr(&ds->sort_status, bad);
}

// Group of particle i from the offsets (binary search: last g with offsets[g] <= i).
__device__ __forceinline__ int group_of(const int64_t *__restrict__ offsets, int64_t n_groups,
                                        int64_t i)
{
    int64_t lo = 0, hi = n_groups - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (offsets[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return (int)lo;
}

__global__ void k_keys_open(int64_t n, const double *__restrict__ pos,
                            const double *__restrict__ mass, const int64_t *__restrict__ offsets,
                            int64_t n_groups, const SegInfo *__restrict__ segs, KeyLayout kl,
                            uint64_t *__restrict__ key, int32_t *__restrict__ idx, DevState *ds,
                            uint4 *__restrict__ rec)
{
    const int shift = kl.coord_bits - kl.lmax;
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int g = group_of(offsets, n_groups, i);
        const SegInfo &s = segs[g];
        double x = pos[i], y = pos[n + i], z = pos[2 * n + i], m = mass[i];
        if (!(finite_bits(x) && finite_bits(y) && finite_bits(z))) bad |= kBadPosition;
        if (!positive_finite_bits(m)) bad |= kBadMass;
        uint32_t X = fix_open(x, s.origin[0], s.inv_q[0]);
        uint32_t Y = fix_open(y, s.origin[1], s.inv_q[1]);
        uint32_t Z = fix_open(z, s.origin[2], s.inv_q[2]);
        uint64_t k = morton3(X >> shift, Y >> shift, Z >> shift);
        if (kl.seg_bits > 0) k |= (uint64_t)g << (3 * kl.lmax);
        key[i] = k;
        idx[i] = (int32_t)i;
        if (rec) rec[i] = make_uint4(X, Y, Z, __float_as_uint((float)m));
    }
    if (bad) atomicOr(&ds->sort_status, bad);
}

// ---------------------------------------------------------------------------------------
// LSD radix sort, 8-bit digits, over tiles of kTileKeys keys (one block per tile).
// The digit counts of every tile are laid out digit-major, so one exclusive scan gives each
// (digit, tile) its first output position.  The scatter ranks the tile stably: warp w owns
// keys [w*kWarpKeys, (w+1)*kWarpKeys) of the tile and ranks equal digits round by round with
// __match_any_sync; per-warp digit counts then give every key its place in the tile ordered
// by digit.  The tile is reordered in shared memory and written out so that the keys of one
// digit go to consecutive addresses (whole sectors instead of scattered 8-byte writes).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t *__restrict__ key,
                                                             int64_t n, int shift,
                                                             int32_t *__restrict__ hist,
                                                             int64_t n_tiles)
{
    __shared__ int cnt[kRadixBins];
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        cnt[threadIdx.x] = 0;
        __syncthreads();
        const int64_t base = t * kTileKeys;
#pragma unroll 4
        for (int k = 0; k < kKeysPerThread; k++) {
            const int64_t i = base + k * kSortThreads + threadIdx.x;
            if (i < n) atomicAdd(&cnt[(int)((key[i] >> shift) & (kRadixBins - 1))], 1);
        }
        __syncthreads();
        hist[(int64_t)threadIdx.x * n_tiles + t] = cnt[threadIdx.x];
        __syncthreads();
    }
}

struct ScatterSmem {
    uint64_t keys[kTileKeys];                 // the tile in digit order
    int32_t idx[kTileKeys];
    int wcnt[kSortThreads / 32][kRadixBins];  // per-warp digit counts, then their prefix over warps
    int dstart[kRadixBins];                   // first position of each digit in the tile
    int goff[kRadixBins];                     // first output position of each digit of the tile
    int wsum[kSortThreads / 32];
};

__global__ void __launch_bounds__(kSortThreads, 2) k_radix_scatter(
    const uint64_t *__restrict__ key_in, const int32_t *__restrict__ idx_in,
    uint64_t *__restrict__ key_out, int32_t *__restrict__ idx_out, int64_t n, int shift,
    const int32_t *__restrict__ offs, int64_t n_tiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem &S = *reinterpret_cast<ScatterSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const int64_t base = t * kTileKeys;
        const int64_t wbase = base + (int64_t)warp * kWarpKeys;
        for (int e = tid; e < (kSortThreads / 32) * kRadixBins; e += kSortThreads) (&S.wcnt[0][0])[e] = 0;
        uint64_t kv[kKeysPerThread];
        int32_t iv[kKeysPerThread];
        int pos[kKeysPerThread];
#pragma unroll
        for (int k = 0; k < kKeysPerThread; k++) {
            const int64_t i = wbase + k * 32 + lane;
            kv[k] = i < n ? key_in[i] : 0ull;
            iv[k] = i < n ? idx_in[i] : 0;
        }
        __syncthreads();
        // stable rank inside the warp's keys, round by round
#pragma unroll
        for (int k = 0; k < kKeysPerThread; k++) {
            const bool valid = wbase + k * 32 + lane < n;
            const int d = valid ? (int)((kv[k] >> shift) & (kRadixBins - 1)) : kRadixBins + lane;
            const unsigned peers = __match_any_sync(kFull, d);
            const int rank = __popc(peers & lanemask_lt());
            pos[k] = valid ? S.wcnt[warp][d] + rank : 0;
            __syncwarp();
            if (valid && rank == 0) S.wcnt[warp][d] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            // thread = digit: prefix over warps, then the digit starts by a block scan
            const int d = tid;
            int tot = 0;
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; w++) {
                const int c = S.wcnt[w][d];
                S.wcnt[w][d] = tot;
                tot += c;
            }
            const int incl = warp_inclusive_scan(tot);
            if (lane == 31) S.wsum[warp] = incl;
            S.goff[d] = offs[(int64_t)d * n_tiles + t];
            __syncthreads();
            int before = 0;
            for (int w = 0; w < warp; w++) before += S.wsum[w];
            S.dstart[d] = before + incl - tot;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKeysPerThread; k++) {
            if (wbase + k * 32 + lane < n) {
                const int d = (int)((kv[k] >> shift) & (kRadixBins - 1));
                const int p = S.dstart[d] + S.wcnt[warp][d] + pos[k];
                S.keys[p] = kv[k];
                S.idx[p] = iv[k];
            }
        }
        __syncthreads();
        const int valid_n = (int)(n - base < kTileKeys ? n - base : kTileKeys);
        for (int p = tid; p < valid_n; p += kSortThreads) {
            const uint64_t kk = S.keys[p];
            const int d = (int)((kk >> shift) & (kRadixBins - 1));
            const int64_t g = (int64_t)S.goff[d] + (p - S.dstart[d]);
            key_out[g] = kk;
            idx_out[g] = S.idx[p];
        }
        __syncthreads();
    }
}

// FP32 sorts: the sorted fixed-point records are the caller-order records in sorted order.
__global__ void k_gather_rec(int64_t n, const int32_t *__restrict__ idx, const uint4 *__restrict__ rec,
                             uint4 *__restrict__ pfix)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        pfix[p] = rec[idx[p]];
}

__global__ void k_gather_periodic(int64_t n, const double *__restrict__ pos,
                                  const double *__restrict__ mass,
                                  const int32_t *__restrict__ idx, SegInfo seg,
                                  uint4 *__restrict__ pfix, double4_32a *__restrict__ pdbl)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[p];
        double x = pos[i], y = pos[n + i], z = pos[2 * n + i], m = mass[i];
        uint4 f;
        f.x = fix_periodic(x, seg.inv_q[0]);
        f.y = fix_periodic(y, seg.inv_q[1]);
        f.z = fix_periodic(z, seg.inv_q[2]);
        f.w = __float_as_uint((float)m);
        pfix[p] = f;
        pdbl[p] = make_double4_32a(x, y, z, m);
    }
}

__global__ void k_gather_open(int64_t n, const double *__restrict__ pos,
                              const double *__restrict__ mass, const int32_t *__restrict__ idx,
                              const uint64_t *__restrict__ key, const SegInfo *__restrict__ segs,
                              KeyLayout kl, uint4 *__restrict__ pfix, double4_32a *__restrict__ pdbl)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[p];
        const int g = kl.seg_bits > 0 ? (int)(key[p] >> (3 * kl.lmax)) : 0;
        const SegInfo &s = segs[g];
        double x = pos[i], y = pos[n + i], z = pos[2 * n + i], m = mass[i];
        uint4 f;
        f.x = fix_open(x, s.origin[0], s.inv_q[0]);
        f.y = fix_open(y, s.origin[1], s.inv_q[1]);
        f.z = fix_open(z, s.origin[2], s.inv_q[2]);
        f.w = __float_as_uint((float)m);
        pfix[p] = f;
        pdbl[p] = make_double4_32a(x, y, z, m);
    }
}

// Dense start table of each segment at its level_c: tab[c] = first sorted index whose
// level-c cell is >= c, for c = 0 .. 8^level_c (the last entry is the segment end).
__global__ void k_cell_table(int64_t n, const uint64_t *__restrict__ key,
                             const SegInfo *__restrict__ segs, KeyLayout kl,
                             int32_t *__restrict__ tab)
{
    const uint64_t mmask = kl.lmax >= 21 ? 0x7fffffffffffffffull : ((1ull << (3 * kl.lmax)) - 1);
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    // Particle p fills the cells after its predecessor's cell up to its own; the last particle
    // of a segment also fills the cells after its own up to the end marker.  Each cell is
    // written once.  A run of up to kOwnRun cells is written by its lane; longer runs (voids)
    // are written by the whole warp, one run at a time, with consecutive lanes on consecutive
    // cells.  The loop bound is the warp's first index, so the warp stays converged.
    constexpr int64_t kOwnRun = 8;
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n;
         base += n_warps * 32) {
        const int64_t p = base + lane;
        int64_t a = 0, b = -1, a2 = 0, b2 = -1;  // runs [a, b] get p, [a2, b2] get the segment end
        int32_t *t = tab;
        int32_t end = 0;
        if (p < n) {
            const uint64_t k = key[p];
            const int g = kl.seg_bits > 0 ? (int)(k >> (3 * kl.lmax)) : 0;
            const SegInfo &s = segs[g];
            const int sh = 3 * (kl.lmax - s.level_c);
            const int64_t pre = (int64_t)((k & mmask) >> sh);
            const int64_t prev = p == s.start ? -1 : (int64_t)((key[p - 1] & mmask) >> sh);
            t = tab + s.tab_off;
            a = prev + 1;
            b = pre;
            if (p == s.end - 1) {
                a2 = pre + 1;
                b2 = 1ll << (3 * s.level_c);
                end = (int32_t)s.end;
            }
        }
        const bool own1 = b - a < kOwnRun, own2 = b2 - a2 < kOwnRun;
        if (own1)
            for (int64_t c = a; c <= b; c++) t[c] = (int32_t)p;
        if (own2)
            for (int64_t c = a2; c <= b2; c++) t[c] = end;
        for (int r = 0; r < 2; r++) {
            unsigned m = __ballot_sync(kFull, r == 0 ? !own1 : !own2);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                const int64_t ra = __shfl_sync(kFull, r == 0 ? a : a2, src);
                const int64_t rb = __shfl_sync(kFull, r == 0 ? b : b2, src);
                const int32_t rv = __shfl_sync(kFull, r == 0 ? (int32_t)p : end, src);
                int32_t *rt = (int32_t *)__shfl_sync(kFull, (unsigned long long)t, src);
                for (int64_t c = ra + lane; c <= rb; c += 32) rt[c] = rv;
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// Batch groups: bounding boxes, fixed-point frames and table sizes.
// ---------------------------------------------------------------------------------------
__global__ void k_group_setup(int64_t n_groups, const int64_t *__restrict__ offsets,
                              const double *__restrict__ pos, int64_t n,
                              const double *__restrict__ nngb, const double *__restrict__ tol,
                              KeyLayout kl, int table_extra, double self_floor,
                              SegInfo *__restrict__ segs, int32_t *__restrict__ tsize, DevState *ds)
{
    __shared__ double red[6][kSortThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
        const int64_t s = offsets[g], e = offsets[g + 1];
        double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
        for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
#pragma unroll
            for (int d = 0; d < 3; d++) {
                double v = pos[d * n + i];
                lo[d] = fmin(lo[d], v);
                hi[d] = fmax(hi[d], v);
            }
        }
#pragma unroll
        for (int d = 0; d < 3; d++) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo[d] = fmin(lo[d], __shfl_xor_sync(kFull, lo[d], o));
                hi[d] = fmax(hi[d], __shfl_xor_sync(kFull, hi[d], o));
            }
            if (lane == 0) {
                red[d][warp] = lo[d];
                red[3 + d][warp] = hi[d];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            SegInfo si;
            si.box[0] = si.box[1] = si.box[2] = 0.0;
            double ext = 0.0;
            for (int d = 0; d < 3; d++) {
                double a = DBL_MAX, b = -DBL_MAX;
                for (int w = 0; w < kSortThreads / 32; w++) {
                    a = fmin(a, red[d][w]);
                    b = fmax(b, red[3 + d][w]);
                }
                si.origin[d] = e > s ? a : 0.0;
                if (e > s && b - a > ext) ext = b - a;
            }
            if (!(ext > 0.0)) ext = 1.0;
            // a little slack keeps the largest coordinate strictly below 2^31 units
            ext *= 1.0 + 1.0 / 1048576.0;
            const double q = ext / 2147483648.0;
            for (int d = 0; d < 3; d++) {
                si.q[d] = q;
                si.inv_q[d] = 1.0 / q;
            }
            si.nngb = nngb[g];
            si.tol = tol[g];
            si.half_box = HUGE_VAL;
            si.periodic = 0;
            const int64_t cnt = e - s;
            int lc = 0;
            while (lc < kl.lmax - 1 && (1ll << (3 * (lc + 1))) <= (cnt << (3 * table_extra))) lc++;
            si.level_c = lc;
            si.tab_off = 0;
            si.start = (int32_t)s;
            si.end = (int32_t)e;
            si.pad = 0;
            segs[g] = si;
            tsize[g] = (int32_t)((1ll << (3 * lc)) + 1);
            if (!(si.nngb > self_floor) || !(si.tol >= 0.0) || e < s) atomicOr(&ds->sort_status, kBadH);
        }
        __syncthreads();
    }
}

__global__ void k_group_tab_off(int64_t n_groups, const int32_t *__restrict__ toff,
                                SegInfo *__restrict__ segs)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n_groups;
         g += (int64_t)gridDim.x * blockDim.x)
        segs[g].tab_off = toff[g];
}

int blocks_for(int64_t n, int threads, int cap)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)(b < cap ? b : cap);
}

}  // namespace

int64_t radix_hist_size(int64_t n_max) { return (int64_t)kRadixBins * ((n_max + kTileKeys - 1) / kTileKeys + 1); }

cudaError_t launch_keys_periodic(const SortArgs &a, int64_t n, const double *pos, const double *mass,
                                 const SegInfo &seg, const double box[3], cudaStream_t st, uint4 *rec)
{
    k_keys_periodic<<<blocks_for(n, 256, a.grid_cap), 256, 0, st>>>(
        n, pos, mass, seg, a.kl, box[0], box[1], box[2], a.key[0], a.idx[0], a.ds, rec);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_group_setup(const SortArgs &a, int64_t n_groups, const int64_t *offsets,
                               const double *pos, int64_t n, const double *nngb, const double *tol,
                               int32_t *tsize, int32_t *toff, cudaStream_t st)
{
    k_group_setup<<<blocks_for(n_groups, 1, a.grid_cap), kSortThreads, 0, st>>>(
        n_groups, offsets, pos, n, nngb, tol, a.kl, a.table_extra, a.self_floor, a.segs, tsize, a.ds);
    if (a.launches) *a.launches += 1;
    cudaError_t e = scan_exclusive(tsize, toff, n_groups, nullptr, nullptr, a.scan_aux, a.grid_cap, st,
                                   a.launches);
    if (e != cudaSuccess) return e;
    k_group_tab_off<<<blocks_for(n_groups, 256, a.grid_cap), 256, 0, st>>>(n_groups, toff, a.segs);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_keys_open(const SortArgs &a, int64_t n, const double *pos, const double *mass,
                             const int64_t *offsets, int64_t n_groups, cudaStream_t st, uint4 *rec)
{
    k_keys_open<<<blocks_for(n, 256, a.grid_cap), 256, 0, st>>>(n, pos, mass, offsets, n_groups,
                                                                  a.segs, a.kl, a.key[0], a.idx[0],
                                                                  a.ds, rec);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

// Sorts (key[0], idx[0]) in place (ping-pong through key[1]/idx[1]); returns the buffer
// index holding the result in *which.
cudaError_t launch_radix_sort(const SortArgs &a, int64_t n, int *which, cudaStream_t st)
{
    const int64_t n_tiles = (n + kTileKeys - 1) / kTileKeys;
    const int grid = blocks_for(n_tiles, 1, a.grid_cap);
    const int smem = (int)sizeof(ScatterSmem);
    cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int cur = 0;
    for (int shift = 0; shift < a.kl.key_bits; shift += kRadixBits) {
        k_radix_hist<<<grid, kSortThreads, 0, st>>>(a.key[cur], n, shift, a.hist, n_tiles);
        if (a.launches) *a.launches += 1;
        cudaError_t e = scan_exclusive(a.hist, a.hist_off, (int64_t)kRadixBins * n_tiles, nullptr, nullptr,
                                       a.scan_aux, a.grid_cap, st, a.launches);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<grid, kSortThreads, smem, st>>>(a.key[cur], a.idx[cur], a.key[1 - cur],
                                                          a.idx[1 - cur], n, shift, a.hist_off, n_tiles);
        if (a.launches) *a.launches += 1;
        cur = 1 - cur;
    }
    *which = cur;
    return cudaGetLastError();
}

cudaError_t launch_gather_periodic(const SortArgs &a, int64_t n, const double *pos,
                                   const double *mass, const int32_t *idx, const SegInfo &seg,
                                   cudaStream_t st)
{
    k_gather_periodic<<<blocks_for(n, 256, a.grid_cap), 256, 0, st>>>(n, pos, mass, idx, seg, a.pfix,
                                                                       a.pdbl);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_open(const SortArgs &a, int64_t n, const double *pos, const double *mass,
                               const int32_t *idx, const uint64_t *key, cudaStream_t st)
{
    k_gather_open<<<blocks_for(n, 256, a.grid_cap), 256, 0, st>>>(n, pos, mass, idx, key, a.segs, a.kl,
                                                                   a.pfix, a.pdbl);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather_rec(const SortArgs &a, int64_t n, const int32_t *idx, const uint4 *rec,
                              cudaStream_t st)
{
    k_gather_rec<<<blocks_for(n, 256, a.grid_cap), 256, 0, st>>>(n, idx, rec, a.pfix);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_cell_table(const SortArgs &a, int64_t n, const uint64_t *key, cudaStream_t st)
{
    k_cell_table<<<blocks_for(n, 256, a.grid_cap), 256, 0, st>>>(n, key, a.segs, a.kl, a.ctab);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

}  // namespace sph
