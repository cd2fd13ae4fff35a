// sph_density.cu -- the density pass: neighbour search + kernel sums for every target on
// the todo list (Eq. 1 with the M4 or Wendland C6 kernel; the density loop of Listing 1).
//
// Work decomposition.  The todo list (sorted positions of unconverged particles, in Morton
// order) is cut into work items of up to 32 consecutive targets that share an octree cell
// (sph_solve.cu).  A persistent grid of warps pops items from a device counter (the dynamic
// scheduling of Listing 3, without a lock).  Per item, the warp:
//   1. builds the item's query box Q = bounding box of the targets grown by h_max, in
//      32-bit fixed point relative to the first target, and a ball around the targets' box
//      centre that every in-h candidate lies in (sph_items.cuh);
//   2. picks the octree level whose cells are at least |Q|/cell_div, skips the cells that
//      lie outside the ball, and looks up each remaining cell's particle range (dense table
//      at or above the table level, binary search on the sorted keys below it);
//   3. streams all those cells as one list with coalesced 16-byte loads, keeps the particles
//      inside Q and the ball (ballot compaction) and stages them in shared memory as FP32
//      offsets from the first target (formed exactly in integer arithmetic, rounded once);
//   4. runs the pair loop: lanes are (target, slice) pairs over the staged candidates.
// FP32 path: each lane tests two candidates at a time with two-wide FP32 instructions and
// evaluates the kernel under the r < h test; partial sums enter compensated (Kahan)
// accumulators every 32 steps.
// FP64 path: the staged FP32 offsets only pre-filter with a widened radius; every pair that
// passes is recomputed from the FP64 positions exactly as the FP64 reference formulae are
// written (IEEE roundings, no contraction), so neighbour sets and per-pair terms are the
// FP64 ones.
#include <climits>

#include "sph_items.cuh"
#include "sph_kernels.cuh"

namespace sph {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kStage = 256;            // candidates staged per warp before a pair-loop flush
constexpr int kStageCap = kStage + 32; // + room to pad the stage to a multiple of 32
constexpr int kRing = 32;              // per-lane queue of in-h pairs (power of two)
constexpr int kSubSteps = 16;          // tests per lane between drains (<= kRing / 2)
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

struct Acc32 {
    float s_mw, c_mw, s_w, c_w, s_dw, c_dw;  // compensated totals
    float p_mw, p_w, p_dw;                   // plain partial sums since the last merge
    int count;
};

__device__ __forceinline__ void merge32(Acc32 &A)
{
    kahan_add(A.s_mw, A.c_mw, A.p_mw);
    kahan_add(A.s_w, A.c_w, A.p_w);
    kahan_add(A.s_dw, A.c_dw, A.p_dw);
    A.p_mw = A.p_w = A.p_dw = 0.f;
}

// The M4 shape as a B-spline with u = max(1-q, 0) and v = max(1-2q, 0):
//   w = 2 u^3 - v^3,   -q w' = 6 q (u^2 - v^2),
// both zero for q >= 1, with no branch on q.  The sums carry w/2 and -q w'/6; the factors
// 2 and 6 are applied once per target.
// kInside: the caller already knows q < 1 (up to one rounding), so u needs no clamp.
template <bool kInside = false>
__device__ __forceinline__ void m4_half(float q, float &w_half, float &dw_sixth)
{
    const float u = kInside ? 1.f - q : fmaxf(1.f - q, 0.f);
    const float v = fmaxf(fmaf(-2.f, q, 1.f), 0.f);
    const float u2 = u * u, v2 = v * v;
    w_half = fmaf(-0.5f * v, v2, u2 * u);
    dw_sixth = q * (u2 - v2);
}

// The Wendland C6 shape with u = max(1-q, 0):
//   w = u^8 (1 + 8q + 25q^2 + 32q^3),   -q w' = 22 q^2 u^7 (1 + 7q + 16q^2);
// the sums carry w and -q w'/22.
template <bool kInside = false>
__device__ __forceinline__ void c6_shape(float q, float &w, float &dw_22)
{
    const float u = kInside ? 1.f - q : fmaxf(1.f - q, 0.f);
    const float u2 = u * u, u4 = u2 * u2;
    const float u7 = u4 * u2 * u, u8 = u4 * u4;
    w = u8 * fmaf(q, fmaf(q, fmaf(q, 32.f, 25.f), 8.f), 1.f);
    dw_22 = (q * q) * u7 * fmaf(q, fmaf(q, 16.f, 7.f), 1.f);
}

// kKern: 0 = M4 cubic spline, 1 = Wendland C6
template <int kKern, bool kInside = false>
__device__ __forceinline__ void shape32(float q, float &w, float &dw)
{
    if (kKern == 0) m4_half<kInside>(q, w, dw);
    else c6_shape<kInside>(q, w, dw);
}

// One in-h pair in FP32 from its squared distance and the neighbour mass.
template <int kKern>
__device__ __forceinline__ void pair32(float2 e, float hinv2, Acc32 &A)
{
    const float q = sqrt_approx(e.x * hinv2);
    float w, dw;
    shape32<kKern>(q, w, dw);
    A.p_mw = fmaf(e.y, w, A.p_mw);
    A.p_w += w;
    A.p_dw += dw;
    A.count++;
}

// ---- FP64 pair terms, written as the FP64 reference writes them --------------------------
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

__device__ __forceinline__ double w64_c6(double q)
{
    if (q < 1.0) {
        const double a = __dsub_rn(1.0, q);
        const double a2 = __dmul_rn(a, a);
        const double a4 = __dmul_rn(a2, a2);
        const double a8 = __dmul_rn(a4, a4);
        const double p = __dadd_rn(1.0, __dmul_rn(q, __dadd_rn(8.0, __dmul_rn(q, __dadd_rn(25.0, __dmul_rn(q, 32.0))))));
        return __dmul_rn(a8, p);
    }
    return 0.0;
}

__device__ __forceinline__ double mqdw64_c6(double q)
{
    if (q < 1.0) {
        const double a = __dsub_rn(1.0, q);
        const double a2 = __dmul_rn(a, a);
        const double a4 = __dmul_rn(a2, a2);
        const double a7 = __dmul_rn(__dmul_rn(a4, a2), a);
        const double p = __dadd_rn(1.0, __dmul_rn(q, __dadd_rn(7.0, __dmul_rn(q, 16.0))));
        return __dmul_rn(__dmul_rn(__dmul_rn(22.0, __dmul_rn(q, q)), a7), p);
    }
    return 0.0;
}

struct Acc64 {
    double s_mw, s_w, s_dw;
    int count;
};

template <int kKern>
__device__ __forceinline__ bool pair64(const double4_32a &ti, const double4_32a &cj, double h,
                                       double h2, const SegInfo &S, Acc64 &A)
{
    double dx = __dsub_rn(cj.x, ti.x);
    double dy = __dsub_rn(cj.y, ti.y);
    double dz = __dsub_rn(cj.z, ti.z);
    if (S.periodic) {
        dx = min_image64(dx, S.box[0]);
        dy = min_image64(dy, S.box[1]);
        dz = min_image64(dz, S.box[2]);
    }
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (r2 < h2) {
        const double q = __ddiv_rn(__dsqrt_rn(r2), h);
        const double w = kKern == 0 ? w64(q) : w64_c6(q);
        A.s_mw = __dadd_rn(A.s_mw, __dmul_rn(cj.w, w));
        A.s_w = __dadd_rn(A.s_w, w);
        A.s_dw = __dadd_rn(A.s_dw, kKern == 0 ? mqdw64(q) : mqdw64_c6(q));
        A.count++;
        return true;
    }
    return false;
}

// Neighbour export: one in-h pair of a sampled target (sorted position j of the neighbour).
__device__ __forceinline__ void nb_record(const SolveArgs &a, int slot, int j)
{
    const int c = atomicAdd(&a.nb_cnt[slot], 1);
    if (c < a.nb_max) a.nb_out[(int64_t)slot * a.nb_max + c] = a.idx[j];
}

// Auxiliary work of a density-kernel instantiation: none, the neighbour export of sampled
// targets, or the recording of every target's cached neighbour list.
constexpr int kAuxNone = 0, kAuxExport = 1, kAuxRecord = 2;

// Per-lane geometry of the pair loop: lane = (target t, slice s); the lane tests staged
// candidates s, s + slices, s + 2 slices, ... against target t.
struct LaneTarget {
    float tx, ty, tz;  // target offset from the item origin
    float h2;          // h^2 for the test (FP64 path: widened radius); -1 for idle lanes
    float hinv2;
    int slices, s;
    int sh;            // log2(slices)
    int slot;          // neighbour export: sample row of the target, or -1
    float r2l;         // list recording: squared list radius (FP64: widened); -1 for idle lanes
    int tslot;         // list recording: the target's index in the item
    int p;             // list recording: the target's sorted position
};

// List recording: a candidate (sorted position j) within the list radius of the lane's target.
__device__ __forceinline__ void lst_record(const SolveArgs &a, int *lcnt, const LaneTarget &L, int j)
{
    const int c = atomicAdd(&lcnt[L.tslot], 1);
    if (c < a.list_entries) a.lst[(int64_t)L.p * a.list_entries + c] = j;
}

// Stage layout of the packed FP32 path (kMode 2).  Candidate slot j is tested by slice
// s = j mod S at step k = j / S (S = slices).  Steps 2i and 2i + 1 of one slice share two
// float4s, (x0, x1, y0, y1) and (z0, z1, m0, m1), so a lane loads two candidates as packed
// coordinate pairs and evaluates both with two-wide FP32 instructions.
__device__ __forceinline__ void stage_pair_put(float *__restrict__ st, int j, int sh, float x,
                                               float y, float z, float m)
{
    const int k = j >> sh, s = j & ((1 << sh) - 1);
    float *f = st + ((((k >> 1) << sh) + s) << 3) + (k & 1);
    f[0] = x;
    f[2] = y;
    f[4] = z;
    f[6] = m;
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Two candidates at once, the same roundings as the scalar shape functions: q is clamped
// to at most 1 (q comes from the unclamped r^2 / h^2 of either candidate, padding
// included), so a candidate outside h contributes exactly zero when its partner is inside.
template <int kKern>
__device__ __forceinline__ void shape32x2(float2 q, float2 &w, float2 &dw)
{
    const float2 one = f2(1.f, 1.f), m1 = f2(-1.f, -1.f);
    const float2 u = __ffma2_rn(q, m1, one);  // 1 - q >= 0
    if (kKern == 0) {
        float2 v = __ffma2_rn(q, f2(-2.f, -2.f), one);
        v = f2(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f));
        const float2 u2 = __fmul2_rn(u, u), v2 = __fmul2_rn(v, v);
        w = __ffma2_rn(__fmul2_rn(f2(-0.5f, -0.5f), v), v2, __fmul2_rn(u2, u));
        dw = __fmul2_rn(q, __ffma2_rn(v2, m1, u2));
    } else {
        const float2 u2 = __fmul2_rn(u, u), u4 = __fmul2_rn(u2, u2);
        const float2 u7 = __fmul2_rn(__fmul2_rn(u4, u2), u), u8 = __fmul2_rn(u4, u4);
        const float2 p3 =
            __ffma2_rn(q, __ffma2_rn(q, __ffma2_rn(q, f2(32.f, 32.f), f2(25.f, 25.f)), f2(8.f, 8.f)), one);
        const float2 p2 = __ffma2_rn(q, __ffma2_rn(q, f2(16.f, 16.f), f2(7.f, 7.f)), one);
        w = __fmul2_rn(u8, p3);
        dw = __fmul2_rn(__fmul2_rn(__fmul2_rn(q, q), u7), p2);
    }
}

// Test all staged candidates, queue the in-h ones per lane (ring of kRing entries), and
// evaluate them in warp-wide rounds.  Only rounds in which every lane has a queued pair run
// while testing continues; lanes drain their own backlog once it could overflow, and at
// the end.  This keeps the long pair body on (nearly) full warps however unevenly the
// in-h pairs fall across the targets.
// kMode: 0 = FP64 (queue), 1 = FP32 with the queue until the in-h share is known, 2 = FP32
// evaluated directly (no queue, no ring memory).
// kAux: kAuxExport also records the in-h candidates of sampled targets, kAuxRecord the
// candidates within the list radius of every target (sidx then holds every staged candidate's
// sorted position in linear slot order).
template <int kMode, int kKern, int kAux>
__device__ __forceinline__ void flush(float4 *__restrict__ stage, const int *__restrict__ sidx,
                                      void *__restrict__ ring_raw, int cnt, int direct_pct,
                                      const LaneTarget &L,
                                      Acc32 &A32, Acc64 &A64, const double4_32a &ti, double h,
                                      double h2, const SegInfo &S,
                                      const double4_32a *__restrict__ pdbl, const SolveArgs &a,
                                      int *__restrict__ lcnt)
{
    constexpr bool kF64 = kMode == 0;
    constexpr bool kQueue = kMode < 2;
    const int lane = lane_id();
    if (kMode >= 2) {
        // pad to a multiple of 2 S (an even number of steps per slice) with candidates that
        // are never within h
        const int pad = (cnt + (2 << L.sh) - 1) & ~((2 << L.sh) - 1);
        for (int j = cnt + lane; j < pad; j += 32)
            stage_pair_put((float *)stage, j, L.sh, 3e18f, 3e18f, 3e18f, 0.f);
        __syncwarp();
        const int npair = pad >> (L.sh + 1);
        const float2 ntx = f2(-L.tx, -L.tx), nty = f2(-L.ty, -L.ty), ntz = f2(-L.tz, -L.tz);
        const float2 hinv2 = f2(L.hinv2, L.hinv2);
        const float4 *__restrict__ st4 = stage + 2 * L.s;
        for (int ib = 0; ib < npair; ib += 32) {
            const int ie = ib + 32 < npair ? ib + 32 : npair;
            float2 pmw = f2(0.f, 0.f), pw = pmw, pdw = pmw, pc = pmw;
            // unrolled twice: measured faster than four times on the warm replay and the batch
#pragma unroll 2
            for (int i = ib; i < ie; i++) {
                const float4 A = st4[2 * (i << L.sh)], B = st4[2 * (i << L.sh) + 1];
                const float2 dx = __fadd2_rn(f2(A.x, A.y), ntx);
                const float2 dy = __fadd2_rn(f2(A.z, A.w), nty);
                const float2 dz = __fadd2_rn(f2(B.x, B.y), ntz);
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                const bool in0 = r2.x < L.h2, in1 = r2.y < L.h2;
                if constexpr (kAux == kAuxExport) {
                    if (L.slot >= 0) {
                        // slots of steps 2i and 2i + 1 of this lane's slice
                        const int j0 = ((2 * i) << L.sh) + L.s, j1 = j0 + (1 << L.sh);
                        if (in0 && j0 < cnt) nb_record(a, L.slot, sidx[j0]);
                        if (in1 && j1 < cnt) nb_record(a, L.slot, sidx[j1]);
                    }
                }
                if constexpr (kAux == kAuxRecord) {
                    // padding candidates (3e18) are never within the list radius
                    const int j0 = ((2 * i) << L.sh) + L.s, j1 = j0 + (1 << L.sh);
                    if (r2.x < L.r2l) lst_record(a, lcnt, L, sidx[j0]);
                    if (r2.y < L.r2l) lst_record(a, lcnt, L, sidx[j1]);
                }
                // kMode 2: the pair body runs when either candidate is within h, so a step in
                // which no lane has one costs only the test; kMode 3: branch-free, the
                // unrolled bodies interleave (candidates outside h add exactly zero)
                if (kMode == 3 || in0 || in1) {
                    pc = __fadd2_rn(pc, f2(in0 ? 1.f : 0.f, in1 ? 1.f : 0.f));
                    const float2 x = __fmul2_rn(r2, hinv2);
                    const float2 q = f2(fminf(sqrt_approx(x.x), 1.f), fminf(sqrt_approx(x.y), 1.f));
                    float2 w, dw;
                    shape32x2<kKern>(q, w, dw);
                    pmw = __ffma2_rn(f2(B.z, B.w), w, pmw);
                    pw = __fadd2_rn(pw, w);
                    pdw = __fadd2_rn(pdw, dw);
                }
            }
            // at most 32 terms per partial sum, as in the scalar paths
            A32.p_mw = pmw.x + pmw.y;
            A32.p_w = pw.x + pw.y;
            A32.p_dw = pdw.x + pdw.y;
            A32.count += (int)(pc.x + pc.y);
            merge32(A32);
        }
        __syncwarp();
        return;
    }
    // pad to a multiple of 32 with candidates that are never within h
    const int pad = (cnt + 31) & ~31;
    for (int j = cnt + lane; j < pad; j += 32) stage[j] = make_float4(3e18f, 3e18f, 3e18f, 0.f);
    __syncwarp();
    float2(*ring32)[32] = (float2(*)[32])ring_raw;
    int(*ring64)[32] = (int(*)[32])ring_raw;
    auto drain_one = [&](int &head) {
        if (kF64) {
            const int j = ring64[head & (kRing - 1)][lane];
            const bool in = pair64<kKern>(ti, pdbl[sidx[j]], h, h2, S, A64);
            if (kAux == kAuxExport && in && L.slot >= 0) nb_record(a, L.slot, sidx[j]);
        } else {
            pair32<kKern>(ring32[head & (kRing - 1)][lane], L.hinv2, A32);
        }
        head++;
    };
    const int steps = pad / L.slices;
    int head = 0, tail = 0;
    bool direct = !kQueue;
    int k0 = 0;
    for (; kQueue && k0 < steps && !direct; k0 += kSubSteps) {
        const int k1 = k0 + kSubSteps < steps ? k0 + kSubSteps : steps;
#pragma unroll 4
        for (int k = k0; k < k1; k++) {
            const int j = k * L.slices + L.s;
            const float4 c = stage[j];
            const float dx = c.x - L.tx, dy = c.y - L.ty, dz = c.z - L.tz;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (kAux == kAuxRecord && r2 < L.r2l) lst_record(a, lcnt, L, sidx[j]);
            if (r2 < L.h2) {
                if (kF64) ring64[tail & (kRing - 1)][lane] = j;
                else ring32[tail & (kRing - 1)][lane] = make_float2(r2, c.w);
                tail++;
            }
        }
        // idle lanes never queue anything, so they do not hold the full rounds back
        if (!kF64 && k0 == 0 && k1 == kSubSteps) {
            // most of the first tests were in h: the remaining candidates are evaluated
            // directly (the test and the pair body on all lanes, no queue)
            const int queued = __reduce_add_sync(kFull, L.h2 >= 0.f ? tail : 0);
            const int lanes = __popc(__ballot_sync(kFull, L.h2 >= 0.f));
            direct = direct_pct == 0 || queued * 100 > direct_pct * lanes * kSubSteps;
        }
        const int full = __reduce_min_sync(kFull, L.h2 >= 0.f ? tail - head : INT_MAX);
        // a lane only ever reads ring entries it wrote itself (idle lanes have none)
        for (int r = 0; r < full; r++)
            if (tail - head > 0) drain_one(head);
        const int mx = __reduce_max_sync(kFull, tail - head);
        for (int r = kRing - kSubSteps; r < mx; r++)
            if (tail - head > kRing - kSubSteps) drain_one(head);
        if (!kF64) merge32(A32);
    }
    if (kQueue) {
        const int mx = __reduce_max_sync(kFull, tail - head);
        for (int r = 0; r < mx; r++)
            if (tail - head > 0) drain_one(head);
        if (!kF64) merge32(A32);
    }
    if (!kF64 && direct) {
        for (int kb = k0; kb < steps; kb += 32) {
            const int ke = kb + 32 < steps ? kb + 32 : steps;
#pragma unroll 4
            for (int k = kb; k < ke; k++) {
                const float4 c = stage[k * L.slices + L.s];
                const float dx = c.x - L.tx, dy = c.y - L.ty, dz = c.z - L.tz;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                // the pair body runs under the test: a step in which no lane is within h
                // costs only the test
                if (r2 < L.h2) {
                    const float q = sqrt_approx(r2 * L.hinv2);
                    float w, dw;
                    shape32<kKern, true>(q, w, dw);
                    A32.p_mw = fmaf(c.w, w, A32.p_mw);
                    A32.p_w += w;
                    A32.p_dw += dw;
                    A32.count++;
                }
            }
            merge32(A32);
        }
    }
    __syncwarp();
}

// Per-warp shared memory: the stage, the mode's queue memory, then the item's cell table
// (exclusive prefix of the cell sizes and first particle of every cell).
// The neighbour export and the list recording add the staged candidates' sorted positions to
// the FP32 modes; the recording also keeps one counter per target of the item.
template <int kMode, int kAux = kAuxNone>
__host__ __device__ constexpr int warp_cell_offset()
{
    return kStageCap * 16 + (kMode == 0   ? kStageCap * 4 + kRing * 32 * 4
                             : kMode == 1 ? kRing * 32 * 8
                             : kAux != 0  ? kStageCap * 4
                                          : 0);
}

template <int kMode, int kAux = kAuxNone>
__host__ __device__ constexpr int warp_smem_bytes()
{
    return warp_cell_offset<kMode, kAux>() + 2 * kMaxCells * 4 + (kAux == kAuxRecord ? 32 * 4 : 0);
}

template <int kMode, int kKern, int kAux = kAuxNone>
__global__ void __launch_bounds__(kThreads, kMode >= 2 ? 3 : 2)
    k_density(SolveArgs a, const int32_t *__restrict__ todo)
{
    constexpr bool kF64 = kMode == 0;
    constexpr bool kExp = kAux == kAuxExport;
    constexpr bool kRec = kAux == kAuxRecord;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + (size_t)warp * warp_smem_bytes<kMode, kAux>();
    float4 *stage = (float4 *)wbase;
    int *sidx = (int *)(wbase + kStageCap * 16);
    void *ring = wbase + kStageCap * 16 + (kF64 ? kStageCap * 4 : 0);
    int *cpre = (int *)(wbase + warp_cell_offset<kMode, kAux>());
    int *cbeg = cpre + kMaxCells;
    int *lcnt = cbeg + kMaxCells;  // list recording: candidates recorded per target of the item
    // the branched (2) and branch-free (3) FP32 kernels are both launched when the pass may use
    // either; the one the pass did not choose returns at once
    if (kMode >= 2 && a.free_first && (a.ds->free_now != 0) != (kMode == 3)) return;
    const int n_items = a.ds->n_items;
    const int todo_count = a.ds->dens_count;
    const int pass = a.ds->pass;
    unsigned long long pairs = 0, tests = 0;

    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&a.ds->item_head, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;
        const int t0 = a.items[it];
        const int t1 = it + 1 < n_items ? a.items[it + 1] : todo_count;
        const int G = t1 - t0;
        if (G < 1 || G > 32) {  // the item rules never make one; report, never overrun
            if (lane == 0) atomicOr(&a.ds->status, 8);
            continue;
        }
        int Gp = 1;
        while (Gp < G) Gp <<= 1;
        LaneTarget L;
        L.slices = 32 / Gp;
        L.sh = 5 - (31 - __clz(Gp));
        const int t = lane & (Gp - 1);
        L.s = lane / Gp;
        const bool active = t < G;
        const int p = todo[t0 + (active ? t : 0)];
        L.slot = kExp && active ? a.nb_slot[a.idx[p]] : -1;
        L.tslot = t;
        L.p = p;
        const uint4 P = a.pfix[p];
        const double hd = kF64 ? a.h[p] : 0.0;
        const float hf = kF64 ? (float)hd : a.h32[p];
        const int g = a.kl.seg_bits > 0 ? (int)(a.key[p] >> (3 * a.kl.lmax)) : 0;
        const SegInfo &S = a.segs[g];

        ItemGeom G3;
        int rel[3];
        // when recording lists, the staging region (box and ball) must hold every candidate
        // within the list radius of every target, not only within its h
        const float hq = !kRec ? hf
                         : kF64 ? (float)(hd * (double)a.list_margin) * (1.0f + 1e-5f)
                                : hf * a.list_margin * (1.0f + 1e-5f);
        item_setup(S, a.kl, a.cell_div, active, P, hq, G3, rel);
        const float qf[3] = {(float)S.q[0], (float)S.q[1], (float)S.q[2]};
        const ItemBall B = item_recentre(G3, rel, qf);
        const float ccx = B.cc[0], ccy = B.cc[1], ccz = B.cc[2], ball2 = B.ball2;
        L.tx = (float)rel[0] * qf[0];
        L.ty = (float)rel[1] * qf[1];
        L.tz = (float)rel[2] * qf[2];
        L.hinv2 = 1.0f / (hf * hf);
        double4_32a ti = make_double4_32a(0, 0, 0, 0);
        if (kF64) {
            // widened pre-filter radius: the FP32 offsets and the fixed-point quantisation both
            // stay far inside the margin; the exact FP64 test decides
            const double qmax = fmax(S.q[0], fmax(S.q[1], S.q[2]));
            const float hl = (float)(hd * (1.0 + 1e-4) + 4.0 * qmax);
            L.h2 = active ? hl * hl : -1.f;
            ti = a.pdbl[p];
            if (kRec) {
                const float rl = (float)(hd * a.list_margin * (1.0 + 1e-4) + 4.0 * qmax);
                L.r2l = active ? rl * rl : -1.f;
            }
        } else {
            L.h2 = active ? hf * hf : -1.f;
            if (kRec) {
                const float rl = hf * a.list_margin;
                L.r2l = active ? rl * rl : -1.f;
            }
        }
        if (kRec) {
            __syncwarp();  // the previous item's counters have been read
            if (active && L.s == 0) lcnt[t] = 0;
            __syncwarp();
        }

        const int ncell = G3.nc[0] * G3.nc[1] * G3.nc[2];
        if (ncell > kMaxCells) {  // cannot happen by construction; report, never overrun
            if (lane == 0) atomicOr(&a.ds->status, 8);
            continue;
        }
        long long rr[2];
        item_ranges(G3, g, S, a.kl, a.ctab, a.key, ncell, B.cc0, ball2, qf, rr);

        Acc32 A32 = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
        Acc64 A64 = {0.0, 0.0, 0.0, 0};
        int cnt = 0;
        int staged = 0;
        int total = 0;
        // The item's cells (lane holds cells lane and lane + 32) are streamed as one list in
        // cell order: an exclusive prefix of the cell sizes maps position f of the list to
        // particle cbeg[c] + f - cpre[c] of the last cell c with cpre[c] <= f.  Cells past
        // ncell are empty, so every position maps into a real cell.  Each lane's positions
        // only grow, so it keeps its current cell (index offset, start of the next cell) in
        // registers and searches the table only when it passes into another cell.
        {
            const int b0 = (int)(rr[0] & 0xffffffffll), n0 = (int)(rr[0] >> 32) - b0;
            const int b1 = (int)(rr[1] & 0xffffffffll), n1 = (int)(rr[1] >> 32) - b1;
            const int i0 = warp_inclusive_scan(n0), i1 = warp_inclusive_scan(n1);
            const int tot0 = __shfl_sync(kFull, i0, 31);
            total = tot0 + __shfl_sync(kFull, i1, 31);
            __syncwarp();  // the previous item's reads of the table are done
            cpre[lane] = i0 - n0;
            cbeg[lane] = b0;
            cpre[lane + 32] = tot0 + i1 - n1;
            cbeg[lane + 32] = b1;
            __syncwarp();
        }
        int cc = 0, coff = cbeg[0], cnxt = cpre[1];
        for (int base = 0; base < total; base += 64) {
            // two independent 16-byte loads per lane before either is used
            int jj[2];
            uint4 PP[2];
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int f = base + 32 * half + lane;
                if (f < total && cnxt <= f) {
                    int c = cc;
#pragma unroll
                    for (int step = kMaxCells / 2; step > 0; step >>= 1)
                        if (c + step < kMaxCells && cpre[c + step] <= f) c += step;
                    cc = c;
                    coff = cbeg[c] - cpre[c];
                    cnxt = c + 1 < kMaxCells ? cpre[c + 1] : INT_MAX;
                }
                jj[half] = f < total ? f + coff : -1;
                PP[half] = make_uint4(0, 0, 0, 0);
                if (jj[half] >= 0) PP[half] = a.pfix[jj[half]];
            }
#pragma unroll
            for (int half = 0; half < 2; half++) {
                const int j = jj[half];
                const uint4 &Pj = PP[half];
                int rj[3] = {0, 0, 0};
                bool in = j >= 0 && in_query(G3, Pj, rj);
                float fx = 0.f, fy = 0.f, fz = 0.f;
                if (in) {
                    fx = (float)rj[0] * qf[0];
                    fy = (float)rj[1] * qf[1];
                    fz = (float)rj[2] * qf[2];
                    const float ex = fx - ccx, ey = fy - ccy, ez = fz - ccz;
                    in = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= ball2;
                }
                const unsigned m = __ballot_sync(kFull, in);
                if (in) {
                    const int slot = cnt + __popc(m & lanemask_lt());
                    if (kMode >= 2) stage_pair_put((float *)stage, slot, L.sh, fx, fy, fz, __uint_as_float(Pj.w));
                    else stage[slot] = make_float4(fx, fy, fz, __uint_as_float(Pj.w));
                    if (kF64 || kAux != kAuxNone) sidx[slot] = j;
                }
                cnt += __popc(m);
                if (cnt > kStage - 32) {
                    __syncwarp();
                    flush<kMode, kKern, kAux>(stage, sidx, ring, cnt, a.direct_pct, L, A32, A64, ti, hd,
                                              hd * hd, S, a.pdbl, a, lcnt);
                    staged += cnt;
                    cnt = 0;
                }
            }
        }
        __syncwarp();
        if (cnt > 0) {
            flush<kMode, kKern, kAux>(stage, sidx, ring, cnt, a.direct_pct, L, A32, A64, ti, hd, hd * hd,
                                      S, a.pdbl, a, lcnt);
            staged += cnt;
        }

        // combine the slices of each target
        int count = kF64 ? A64.count : A32.count;
        if constexpr (kF64) {
            double smw = A64.s_mw, sw = A64.s_w, sdw = A64.s_dw;
            for (int o = Gp; o < 32; o <<= 1) {
                smw += __shfl_xor_sync(kFull, smw, o);
                sw += __shfl_xor_sync(kFull, sw, o);
                sdw += __shfl_xor_sync(kFull, sdw, o);
                count += __shfl_xor_sync(kFull, count, o);
            }
            if (active && L.s == 0) {
                const double h = hd;
                if (kKern == 0) {
                    a.e_rho[p] = smw * (8.0 / (kPi * h * h * h));
                    a.e_nw[p] = (32.0 / 3.0) * sw;
                    a.e_dnw[p] = (32.0 / 3.0) * sdw / h;
                } else {
                    a.e_rho[p] = smw * (1365.0 / (64.0 * kPi * h * h * h));
                    a.e_nw[p] = (1365.0 / 48.0) * sw;
                    a.e_dnw[p] = (1365.0 / 48.0) * sdw / h;
                }
                a.e_cnt[p] = count;
                pairs += (unsigned long long)count;
            }
        } else {
            // totals and compensations are combined separately across slices; the compensated
            // totals are then exact to about one FP32 rounding
            float smw = A32.s_mw, cmw = A32.c_mw, sw = A32.s_w, cw = A32.c_w, sdw = A32.s_dw,
                  cdw = A32.c_dw;
            for (int o = Gp; o < 32; o <<= 1) {
                smw += __shfl_xor_sync(kFull, smw, o);
                cmw += __shfl_xor_sync(kFull, cmw, o);
                sw += __shfl_xor_sync(kFull, sw, o);
                cw += __shfl_xor_sync(kFull, cw, o);
                sdw += __shfl_xor_sync(kFull, sdw, o);
                cdw += __shfl_xor_sync(kFull, cdw, o);
                count += __shfl_xor_sync(kFull, count, o);
            }
            if (active && L.s == 0) {
                const float hi = 1.0f / hf;
                // rho = sigma h^-3 sum m w; N_w = (4 pi/3) sigma sum w; dN_w/dh = (4 pi/3) sigma
                // h^-1 sum -q w', with sigma = 8/pi (M4; the sums carry w/2 and -q w'/6) or
                // 1365/(64 pi) (Wendland C6; the sums carry w and -q w'/22)
                const float crho = kKern == 0 ? 2.0f * 2.546479089f : 6.788953041f;
                const float cnw = kKern == 0 ? 2.0f * 10.66666667f : 28.4375f;
                const float cdnw = kKern == 0 ? 6.0f * 10.66666667f : 22.0f * 28.4375f;
                a.e_rho32[p] = crho * (hi * hi * hi) * (smw - cmw);
                a.e_nw32[p] = cnw * (sw - cw);
                a.e_dnw32[p] = cdnw * hi * (sdw - cdw);
                a.e_cnt[p] = count;
                pairs += (unsigned long long)count;
            }
        }
        if (lane == 0) tests += (unsigned long long)staged * (unsigned long long)G;
        if (kRec) {
            // a list holds every candidate within the list radius by the test above, so it serves
            // any later h below that radius (with a margin for the rounding of that test)
            __syncwarp();
            if (active && L.s == 0) {
                const int nrec = lcnt[t];
                const bool fits = nrec <= a.list_entries;
                a.lst_n[p] = fits ? nrec : -1;
                a.lst_r[p] = fits ? (kF64 ? hd * (double)a.list_margin
                                          : (double)(hf * a.list_margin) * (1.0 - 1e-5))
                                  : 0.0;
            }
        }
    }
    pairs = warp_sum(pairs);
    if (lane == 0) {
        if (pairs) {
            atomicAdd(&a.ds->pair_evals, pairs);
            if (pass < kMaxPasses) atomicAdd(&a.ds->pairs_per_pass[pass], pairs);
        }
        if (tests) atomicAdd(&a.ds->pair_tests, tests);
    }
}


// Cached-list pass: the todo targets whose recorded neighbour list still covers their h are
// evaluated from that list, 8 lanes per target and 4 targets per warp; flags[t] = 1 marks the
// targets that must search again (no list, or h beyond the list's radius).  Offsets come from
// the exact 32-bit fixed-point differences of target and neighbour, rounded once to FP32 (FP64
// mode: the FP64 pair exactly as the density pass forms it), so the in-h decisions and pair
// terms are those of Eq. (1) on the list.
constexpr int kListLanes = 8;
constexpr int kListUnroll = 4;

template <bool kF64, int kKern>
__global__ void __launch_bounds__(kThreads) k_list_eval(SolveArgs a, const int32_t *__restrict__ todo)
{
    const int T = a.ds->pass_count;
    const int pass = a.ds->pass;
    const int lane = lane_id(), sub = lane & (kListLanes - 1);
    const int gw = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    constexpr int kPerWarp = 32 / kListLanes;
    unsigned long long pairs = 0, tests = 0, served = 0;
    for (int tb = gw * kPerWarp; tb < T; tb += nw * kPerWarp) {
        const int t = tb + lane / kListLanes;
        const bool have = t < T;
        const int p = have ? todo[t] : 0;
        const double hd = a.h[p];
        const int ln = have ? a.lst_n[p] : -1;
        const bool use = have && ln >= 0 && hd <= a.lst_r[p];
        if (have && sub == 0) a.flags[t] = use ? 0 : 1;
        const int nl = use ? ln : 0;
        const int nmax = __reduce_max_sync(kFull, nl);
        if (nmax == 0) continue;
        const uint4 P = a.pfix[p];
        const int g = a.kl.seg_bits > 0 ? (int)(a.key[p] >> (3 * a.kl.lmax)) : 0;
        const SegInfo &S = a.segs[g];
        const float qx = (float)S.q[0], qy = (float)S.q[1], qz = (float)S.q[2];
        const float hf = kF64 ? (float)hd : a.h32[p];
        const float h2 = hf * hf, hinv2 = 1.0f / (hf * hf);
        const double4_32a ti = kF64 ? a.pdbl[p] : make_double4_32a(0, 0, 0, 0);
        const double hd2 = hd * hd;
        const int32_t *lst = a.lst + (int64_t)p * a.list_entries;
        Acc32 A32 = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
        Acc64 A64 = {0.0, 0.0, 0.0, 0};
        int since = 0;
        for (int k0 = 0; k0 < nmax; k0 += kListLanes * kListUnroll) {
            // the list entries first, then their records, all independent loads
            int jj[kListUnroll];
#pragma unroll
            for (int u = 0; u < kListUnroll; u++) {
                const int k = k0 + kListLanes * u + sub;
                jj[u] = k < nl ? lst[k] : -1;
            }
            if constexpr (kF64) {
                double4_32a C[kListUnroll];
#pragma unroll
                for (int u = 0; u < kListUnroll; u++) C[u] = a.pdbl[jj[u] >= 0 ? jj[u] : p];
#pragma unroll
                for (int u = 0; u < kListUnroll; u++)
                    if (jj[u] >= 0) pair64<kKern>(ti, C[u], hd, hd2, S, A64);
            } else {
                uint4 C[kListUnroll];
#pragma unroll
                for (int u = 0; u < kListUnroll; u++) C[u] = a.pfix[jj[u] >= 0 ? jj[u] : p];
#pragma unroll
                for (int u = 0; u < kListUnroll; u++) {
                    if (jj[u] < 0) continue;
                    const float dx = (float)(int32_t)(C[u].x - P.x) * qx;
                    const float dy = (float)(int32_t)(C[u].y - P.y) * qy;
                    const float dz = (float)(int32_t)(C[u].z - P.z) * qz;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (r2 < h2) {
                        const float q = sqrt_approx(r2 * hinv2);
                        float w, dw;
                        shape32<kKern, true>(q, w, dw);
                        A32.p_mw = fmaf(__uint_as_float(C[u].w), w, A32.p_mw);
                        A32.p_w += w;
                        A32.p_dw += dw;
                        A32.count++;
                    }
                }
                // at most 32 terms per partial sum, as in the density pass
                if (++since == 32 / kListUnroll) {
                    merge32(A32);
                    since = 0;
                }
            }
        }
        if (use && sub == 0) {
            tests += (unsigned long long)ln;
            served++;
        }
        // combine the 8 lanes of each target
        int count = kF64 ? A64.count : A32.count;
        if constexpr (kF64) {
            double smw = A64.s_mw, sw = A64.s_w, sdw = A64.s_dw;
#pragma unroll
            for (int o = kListLanes / 2; o > 0; o >>= 1) {
                smw += __shfl_xor_sync(kFull, smw, o);
                sw += __shfl_xor_sync(kFull, sw, o);
                sdw += __shfl_xor_sync(kFull, sdw, o);
                count += __shfl_xor_sync(kFull, count, o);
            }
            if (use && sub == 0) {
                const double h = hd;
                if (kKern == 0) {
                    a.e_rho[p] = smw * (8.0 / (kPi * h * h * h));
                    a.e_nw[p] = (32.0 / 3.0) * sw;
                    a.e_dnw[p] = (32.0 / 3.0) * sdw / h;
                } else {
                    a.e_rho[p] = smw * (1365.0 / (64.0 * kPi * h * h * h));
                    a.e_nw[p] = (1365.0 / 48.0) * sw;
                    a.e_dnw[p] = (1365.0 / 48.0) * sdw / h;
                }
                a.e_cnt[p] = count;
                pairs += (unsigned long long)count;
            }
        } else {
            merge32(A32);
            float smw = A32.s_mw, cmw = A32.c_mw, sw = A32.s_w, cw = A32.c_w, sdw = A32.s_dw, cdw = A32.c_dw;
#pragma unroll
            for (int o = kListLanes / 2; o > 0; o >>= 1) {
                smw += __shfl_xor_sync(kFull, smw, o);
                cmw += __shfl_xor_sync(kFull, cmw, o);
                sw += __shfl_xor_sync(kFull, sw, o);
                cw += __shfl_xor_sync(kFull, cw, o);
                sdw += __shfl_xor_sync(kFull, sdw, o);
                cdw += __shfl_xor_sync(kFull, cdw, o);
                count += __shfl_xor_sync(kFull, count, o);
            }
            if (use && sub == 0) {
                const float hi = 1.0f / hf;
                const float crho = kKern == 0 ? 2.0f * 2.546479089f : 6.788953041f;
                const float cnw = kKern == 0 ? 2.0f * 10.66666667f : 28.4375f;
                const float cdnw = kKern == 0 ? 6.0f * 10.66666667f : 22.0f * 28.4375f;
                a.e_rho32[p] = crho * (hi * hi * hi) * (smw - cmw);
                a.e_nw32[p] = cnw * (sw - cw);
                a.e_dnw32[p] = cdnw * hi * (sdw - cdw);
                a.e_cnt[p] = count;
                pairs += (unsigned long long)count;
            }
        }
    }
    pairs = warp_sum(pairs);
    tests = warp_sum(tests);
    served = warp_sum(served);
    if (lane == 0) {
        if (pairs) {
            atomicAdd(&a.ds->pair_evals, pairs);
            if (pass < kMaxPasses) atomicAdd(&a.ds->pairs_per_pass[pass], pairs);
        }
        if (tests) atomicAdd(&a.ds->pair_tests, tests);
        if (served) atomicAdd(&a.ds->list_evals, served);
    }
}

}  // namespace

// Every warp works on its own items, so a block is only a bundle of warps: the block size is a
// launch choice (64, 128 or 256 threads, up to the launch bound), with each warp's shared
// memory carved from the block's.
template <int kMode, int kKern>
int blocks_per_sm(int threads)
{
    const int bytes = (threads / 32) * warp_smem_bytes<kMode>();
    // the attribute is set for the largest block, which covers every smaller one
    cudaFuncSetAttribute(k_density<kMode, kKern>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kWarps * warp_smem_bytes<kMode>());
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_density<kMode, kKern>, threads, bytes);
    return b > 0 ? b : 1;
}

int mode_of(int precision, int direct_pct) { return precision == 0 ? 0 : direct_pct == 0 ? 2 : 1; }

int density_blocks_per_sm(int precision, int direct_pct, int threads)
{
    if (threads != 64 && threads != 128) threads = kThreads;
    // both kernels' attributes are set; the grid follows the M4 instantiation (the persistent
    // grid is correct for any size, the work queue balances it)
    switch (mode_of(precision, direct_pct)) {
    case 0: blocks_per_sm<0, 1>(threads); return blocks_per_sm<0, 0>(threads);
    case 1: blocks_per_sm<1, 1>(threads); return blocks_per_sm<1, 0>(threads);
    default:
        blocks_per_sm<3, 1>(threads);
        blocks_per_sm<3, 0>(threads);
        blocks_per_sm<2, 1>(threads);
        return blocks_per_sm<2, 0>(threads);
    }
}

template <int kMode, int kAux = kAuxNone>
void launch_mode(const SolveArgs &a, const int32_t *todo, cudaStream_t st)
{
    const int threads = (a.block_threads == 64 || a.block_threads == 128) ? a.block_threads : kThreads;
    const int bytes = (threads / 32) * warp_smem_bytes<kMode, kAux>();
    if (kAux != kAuxNone) {
        // the auxiliary instantiations are not prepared by density_blocks_per_sm; the persistent
        // grid stays correct whatever number of its blocks are resident at once
        cudaFuncSetAttribute(k_density<kMode, 0, kAux>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kWarps * warp_smem_bytes<kMode, kAux>());
        cudaFuncSetAttribute(k_density<kMode, 1, kAux>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kWarps * warp_smem_bytes<kMode, kAux>());
    }
    if (a.kernel == 0) k_density<kMode, 0, kAux><<<a.density_grid, threads, bytes, st>>>(a, todo);
    else k_density<kMode, 1, kAux><<<a.density_grid, threads, bytes, st>>>(a, todo);
}

template <int kAux>
void launch_modes(const SolveArgs &a, const int32_t *todo, int mode, cudaStream_t st)
{
    if (mode == 0) {
        launch_mode<0, kAux>(a, todo, st);
    } else {
        if (a.free_first) {
            launch_mode<3, kAux>(a, todo, st);
            if (a.launches) *a.launches += 1;
        }
        launch_mode<2, kAux>(a, todo, st);
    }
}

cudaError_t launch_list_eval(const SolveArgs &a, const int32_t *todo, cudaStream_t st)
{
    constexpr int per_block = kThreads / 32 * (32 / kListLanes);
    int64_t blocks = (a.n + per_block - 1) / per_block;
    if (blocks > a.grid_cap) blocks = a.grid_cap;
    if (blocks < 1) blocks = 1;
    const bool f64 = a.precision == 0;
    if (f64 && a.kernel == 0) k_list_eval<true, 0><<<(int)blocks, kThreads, 0, st>>>(a, todo);
    else if (f64) k_list_eval<true, 1><<<(int)blocks, kThreads, 0, st>>>(a, todo);
    else if (a.kernel == 0) k_list_eval<false, 0><<<(int)blocks, kThreads, 0, st>>>(a, todo);
    else k_list_eval<false, 1><<<(int)blocks, kThreads, 0, st>>>(a, todo);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_density(const SolveArgs &a, const int32_t *todo, cudaStream_t st)
{
    const int mode = mode_of(a.precision, a.direct_pct);
    if (a.nb_out || a.lst) {
        // the neighbour export (test aid) and the list recording run the same pass in their own
        // instantiations; the per-lane queue of the non-default FP32 mode 1 has neither
        if (mode == 1) return cudaErrorNotSupported;
        if (a.nb_out) launch_modes<kAuxExport>(a, todo, mode, st);
        else launch_modes<kAuxRecord>(a, todo, mode, st);
        if (a.launches) *a.launches += 1;
        return cudaGetLastError();
    }
    switch (mode) {
    case 0: launch_mode<0>(a, todo, st); break;
    case 1: launch_mode<1>(a, todo, st); break;
    default:
        if (a.free_first) {
            launch_mode<3>(a, todo, st);
            if (a.launches) *a.launches += 1;
        }
        launch_mode<2>(a, todo, st);
        break;
    }
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}


}  // namespace sph
