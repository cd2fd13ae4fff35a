// sph_interact.cu -- the further pair computations of the density loop (Listing 1: after the
// density sum, "other particle interaction computations"; Sec. II-A: the second phase of the
// particle interactions) over the same neighbour sets as Eq. (1), at each particle's h:
//   rho_i      = sum_j m_j W_ij
//   vbar_i     = (1 / rho_i) sum_j m_j W_ij v_j
//   sigma2_i   = (1 / rho_i) sum_j m_j W_ij |v_j - vbar_i|^2
//   (div v)_i  = (1 / rho_i) sum_j m_j (v_j - v_i) . grad_i W_ij
//   (curl v)_i = (1 / rho_i) sum_j m_j (v_i - v_j) x grad_i W_ij
// over j with r_ij < h_i (self included), W_ij = W(r_ij, h_i), grad_i W_ij = dW/dr (r_i - r_j)/r.
//
// The neighbour search is the density pass's: work items of up to 32 consecutive targets, the
// item's query box and ball, its octree cells, coalesced streaming and ballot-compacted staging
// (sph_items.cuh).  Each staged candidate carries its FP32 offset and mass and (FP32 mode) its
// FP32 velocity.  Lanes are (target, slice) pairs over the stage, as in the density pass.
// With u = v_j - v_i, d = r_j - r_i and g(q) = -w'(q)/q (finite at q = 0), every in-h pair adds
// m w, m w u, m w |u|^2, m g (d . u) and m g (d x u) to nine sums; since grad_i W_ij =
// sigma g(q) d / h^5, the outputs are rho = sigma S0 / h^3, vbar = v_i + S1 / S0,
// sigma2 = S2 / S0 - |S1 / S0|^2 (the dispersion about the mean, taken about v_i in one sweep),
// div = D / (h^2 S0) and curl = C / (h^2 S0).
// FP32 mode: FP32 pair terms, plain partial sums of at most 32 terms merged into compensated
// (Kahan) totals, the final combination in FP64.  FP64 mode: the staged FP32 offsets only
// pre-filter with a widened radius; every pair that passes is recomputed from the FP64
// positions and velocities, with the neighbour test formed exactly as the FP64 density pairs
// form it, so the neighbour sets are the FP64 ones.
#include <cfloat>
#include <climits>

#include "sph_items.cuh"
#include "sph_kernels.cuh"

namespace sph {

namespace {

constexpr int kIThreads = 256;
constexpr int kIWarps = kIThreads / 32;
constexpr int kIStage = 128;  // candidates staged per warp before the pair loop runs

template <bool kF64>
__host__ __device__ constexpr int interact_warp_bytes()
{
    // positions + (FP32: velocities | FP64: sorted positions), then the item's cell table
    return kIStage * 16 + kIStage * (kF64 ? 4 : 16) + 2 * kMaxCells * 4;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Shape w(q) and g(q) = -w'(q)/q, FP32, for q in [0, 1].
template <int kKern>
__device__ __forceinline__ void shape_g32(float q, float &w, float &g)
{
    if (kKern == 0) {  // M4: w = 1 - 6 q^2 + 6 q^3 (q <= 1/2), 2 (1 - q)^3
        if (q <= 0.5f) {
            w = fmaf(q * q, fmaf(6.0f, q, -6.0f), 1.0f);
            g = fmaf(-18.0f, q, 12.0f);
        } else {
            const float a = 1.0f - q;
            w = 2.0f * a * a * a;
            g = __fdividef(6.0f * a * a, q);
        }
    } else {  // Wendland C6: w = (1 - q)^8 (1 + 8 q + 25 q^2 + 32 q^3)
        const float a = 1.0f - q, a2 = a * a, a4 = a2 * a2, a7 = a4 * a2 * a;
        w = a7 * a * fmaf(q, fmaf(q, fmaf(q, 32.0f, 25.0f), 8.0f), 1.0f);
        g = 22.0f * a7 * fmaf(q, fmaf(q, 16.0f, 7.0f), 1.0f);
    }
}

template <int kKern>
__device__ __forceinline__ void shape_g64(double q, double &w, double &g)
{
    if (kKern == 0) {
        if (q <= 0.5) {
            w = 1.0 + q * q * (6.0 * q - 6.0);
            g = 12.0 - 18.0 * q;
        } else {
            const double a = 1.0 - q;
            w = 2.0 * a * a * a;
            g = 6.0 * a * a / q;
        }
    } else {
        const double a = 1.0 - q, a2 = a * a, a4 = a2 * a2, a7 = a4 * a2 * a;
        w = a7 * a * (1.0 + q * (8.0 + q * (25.0 + q * 32.0)));
        g = 22.0 * a7 * (1.0 + q * (7.0 + q * 16.0));
    }
}

// The nine sums of one lane: S0, S1 (3), S2, D, C (3).
constexpr int kSums = 9;

struct ISums32 {
    float s[kSums], c[kSums], p[kSums];
    int count;
};

struct ISums64 {
    double s[kSums];
    int count;
};

template <typename T>
__device__ __forceinline__ void add_pair(T (&acc)[kSums], T m, T w, T g, T dx, T dy, T dz, T ux, T uy,
                                         T uz)
{
    const T mw = m * w, mg = m * g;
    acc[0] += mw;
    acc[1] += mw * ux;
    acc[2] += mw * uy;
    acc[3] += mw * uz;
    acc[4] += mw * (ux * ux + uy * uy + uz * uz);
    acc[5] += mg * (dx * ux + dy * uy + dz * uz);
    acc[6] += mg * (dy * uz - dz * uy);
    acc[7] += mg * (dz * ux - dx * uz);
    acc[8] += mg * (dx * uy - dy * ux);
}

struct ILane {
    float tx, ty, tz;  // target offset from the item origin
    float h2;          // FP32 test radius squared (FP64: widened pre-filter); -1 idle lanes
    float hinv2;
    float vx, vy, vz;  // target velocity (FP32 mode)
    int s, slices;     // slice of the stage this lane walks
};

// Pair loop over the staged candidates s, s + slices, ... of this lane.
template <bool kF64, int kKern>
__device__ __forceinline__ void iflush(const float4 *__restrict__ stage, const void *__restrict__ aux,
                                       int cnt, const ILane &L, ISums32 &A32, ISums64 &A64,
                                       const double4_32a &ti, const double4_32a &vi, double hd,
                                       double hd2, const SegInfo &S, const SolveArgs &a,
                                       const InteractArgs &ia)
{
    if (kF64) {
        const int *sidx = (const int *)aux;
        const double4_32a *__restrict__ vrec = (const double4_32a *)ia.vrec;
        for (int k = L.s; k < cnt; k += L.slices) {
            const float4 c = stage[k];
            const float dx = c.x - L.tx, dy = c.y - L.ty, dz = c.z - L.tz;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= L.h2) continue;
            const int j = sidx[k];
            const double4_32a cj = a.pdbl[j];
            double ex = __dsub_rn(cj.x, ti.x), ey = __dsub_rn(cj.y, ti.y), ez = __dsub_rn(cj.z, ti.z);
            if (S.periodic) {
                ex = min_image64(ex, S.box[0]);
                ey = min_image64(ey, S.box[1]);
                ez = min_image64(ez, S.box[2]);
            }
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
            if (!(r2 < hd2)) continue;
            const double q = __ddiv_rn(__dsqrt_rn(r2), hd);
            double w, g;
            shape_g64<kKern>(q, w, g);
            const double4_32a vj = vrec[j];
            add_pair<double>(A64.s, cj.w, w, g, ex, ey, ez, vj.x - vi.x, vj.y - vi.y, vj.z - vi.z);
            A64.count++;
        }
        return;
    }
    const float4 *__restrict__ vst = (const float4 *)aux;
    const int span = 32 * L.slices;  // at most 32 terms per partial sum
    for (int kb = L.s; kb < cnt; kb += span) {
        const int ke = kb + span < cnt ? kb + span : cnt;
#pragma unroll
        for (int i = 0; i < kSums; i++) A32.p[i] = 0.f;
        for (int k = kb; k < ke; k += L.slices) {
            const float4 c = stage[k];
            const float dx = c.x - L.tx, dy = c.y - L.ty, dz = c.z - L.tz;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 < L.h2) {
                const float q = fminf(sqrt_approx(r2 * L.hinv2), 1.0f);
                float w, g;
                shape_g32<kKern>(q, w, g);
                const float4 v = vst[k];
                add_pair<float>(A32.p, c.w, w, g, dx, dy, dz, v.x - L.vx, v.y - L.vy, v.z - L.vz);
                A32.count++;
            }
        }
#pragma unroll
        for (int i = 0; i < kSums; i++) kahan_add(A32.s[i], A32.c[i], A32.p[i]);
    }
}

// Three FP32 blocks per SM (80 registers, a few spilled) hide the staging loads' latency
// better than two without spills (measured 147 against 193 ms on 67M particles).
template <bool kF64, int kKern>
__global__ void __launch_bounds__(kIThreads, kF64 ? 2 : 3) k_interact(SolveArgs a, InteractArgs ia,
                                                        const int32_t *__restrict__ todo)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + (size_t)warp * interact_warp_bytes<kF64>();
    float4 *stage = (float4 *)wbase;
    void *aux = wbase + kIStage * 16;
    int *cpre = (int *)(wbase + kIStage * 16 + kIStage * (kF64 ? 4 : 16));
    int *cbeg = cpre + kMaxCells;
    const int n_items = a.ds->n_items;
    const int todo_count = a.ds->dens_count;
    const int64_t n = a.n;
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
        ILane L;
        L.slices = 32 / Gp;
        const int t = lane & (Gp - 1);
        L.s = lane / Gp;
        const bool active = t < G;
        const int p = todo[t0 + (active ? t : 0)];
        const int64_t i = a.idx[p];
        const uint4 P = a.pfix[p];
        const double hd = a.h[p];
        const float hf = kF64 ? (float)hd : a.h32[p];
        const int g = a.kl.seg_bits > 0 ? (int)(a.key[p] >> (3 * a.kl.lmax)) : 0;
        const SegInfo &S = a.segs[g];

        ItemGeom G3;
        int rel[3];
        item_setup(S, a.kl, a.cell_div, active, P, hf, G3, rel);
        const float qf[3] = {(float)S.q[0], (float)S.q[1], (float)S.q[2]};
        const ItemBall B = item_recentre(G3, rel, qf);
        L.tx = (float)rel[0] * qf[0];
        L.ty = (float)rel[1] * qf[1];
        L.tz = (float)rel[2] * qf[2];
        L.hinv2 = 1.0f / (hf * hf);
        double4_32a ti = make_double4_32a(0, 0, 0, 0), vi = make_double4_32a(0, 0, 0, 0);
        if (kF64) {
            const double qmax = fmax(S.q[0], fmax(S.q[1], S.q[2]));
            const float hl = (float)(hd * (1.0 + 1e-4) + 4.0 * qmax);
            L.h2 = active ? hl * hl : -1.f;
            ti = a.pdbl[p];
            vi = ((const double4_32a *)ia.vrec)[p];
            L.vx = L.vy = L.vz = 0.f;
        } else {
            L.h2 = active ? hf * hf : -1.f;
            const float4 v = ((const float4 *)ia.vrec)[p];
            L.vx = v.x;
            L.vy = v.y;
            L.vz = v.z;
        }
        const int ncell = G3.nc[0] * G3.nc[1] * G3.nc[2];
        if (ncell > kMaxCells) {  // cannot happen by construction; report, never overrun
            if (lane == 0) atomicOr(&a.ds->status, 8);
            continue;
        }
        long long rr[2];
        item_ranges(G3, g, S, a.kl, a.ctab, a.key, ncell, B.cc0, B.ball2, qf, rr);

        ISums32 A32;
        ISums64 A64;
#pragma unroll
        for (int k = 0; k < kSums; k++) {
            A32.s[k] = A32.c[k] = A32.p[k] = 0.f;
            A64.s[k] = 0.0;
        }
        A32.count = A64.count = 0;
        int cnt = 0, staged = 0, total = 0;
        // the cells as one list in cell order (exclusive prefix of their sizes), as in the
        // density pass
        {
            const int b0 = (int)(rr[0] & 0xffffffffll), n0 = (int)(rr[0] >> 32) - b0;
            const int b1 = (int)(rr[1] & 0xffffffffll), n1 = (int)(rr[1] >> 32) - b1;
            const int i0 = warp_inclusive_scan(n0), i1 = warp_inclusive_scan(n1);
            const int tot0 = __shfl_sync(kFull, i0, 31);
            total = tot0 + __shfl_sync(kFull, i1, 31);
            __syncwarp();
            cpre[lane] = i0 - n0;
            cbeg[lane] = b0;
            cpre[lane + 32] = tot0 + i1 - n1;
            cbeg[lane + 32] = b1;
            __syncwarp();
        }
        const double hd2 = hd * hd;
        int cc = 0, coff = cbeg[0], cnxt = cpre[1];
        for (int base = 0; base < total; base += 64) {
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
                int rj[3] = {0, 0, 0};
                bool in = j >= 0 && in_query(G3, PP[half], rj);
                float fx = 0.f, fy = 0.f, fz = 0.f;
                if (in) {
                    fx = (float)rj[0] * qf[0];
                    fy = (float)rj[1] * qf[1];
                    fz = (float)rj[2] * qf[2];
                    const float ex = fx - B.cc[0], ey = fy - B.cc[1], ez = fz - B.cc[2];
                    in = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= B.ball2;
                }
                const unsigned m = __ballot_sync(kFull, in);
                if (in) {
                    const int slot = cnt + __popc(m & lanemask_lt());
                    stage[slot] = make_float4(fx, fy, fz, __uint_as_float(PP[half].w));
                    if (kF64) ((int *)aux)[slot] = j;
                    else ((float4 *)aux)[slot] = ((const float4 *)ia.vrec)[j];
                }
                cnt += __popc(m);
                if (cnt > kIStage - 32) {
                    __syncwarp();
                    iflush<kF64, kKern>(stage, aux, cnt, L, A32, A64, ti, vi, hd, hd2, S, a, ia);
                    __syncwarp();
                    staged += cnt;
                    cnt = 0;
                }
            }
        }
        __syncwarp();
        if (cnt > 0) {
            iflush<kF64, kKern>(stage, aux, cnt, L, A32, A64, ti, vi, hd, hd2, S, a, ia);
            staged += cnt;
        }
        __syncwarp();

        // combine the slices of each target, then the outputs (caller order)
        double T[kSums];
        int count = kF64 ? A64.count : A32.count;
        for (int o = Gp; o < 32; o <<= 1) count += __shfl_xor_sync(kFull, count, o);
        if constexpr (kF64) {
#pragma unroll
            for (int k = 0; k < kSums; k++) {
                double v = A64.s[k];
                for (int o = Gp; o < 32; o <<= 1) v += __shfl_xor_sync(kFull, v, o);
                T[k] = v;
            }
        } else {
            // totals and compensations are combined separately across slices
#pragma unroll
            for (int k = 0; k < kSums; k++) {
                float sv = A32.s[k], cv = A32.c[k];
                for (int o = Gp; o < 32; o <<= 1) {
                    sv += __shfl_xor_sync(kFull, sv, o);
                    cv += __shfl_xor_sync(kFull, cv, o);
                }
                T[k] = (double)sv - (double)cv;
            }
        }
        if (active && L.s == 0) {
            constexpr double kPi = 3.14159265358979323846;
            const double sigma = kKern == 0 ? 8.0 / kPi : 1365.0 / (64.0 * kPi);
            const double S0 = T[0];
            const double m1x = T[1] / S0, m1y = T[2] / S0, m1z = T[3] / S0;
            const double gs = 1.0 / (hd * hd * S0);
            ia.rho[i] = sigma * S0 / (hd * hd * hd);
            ia.vmean[i] = ia.vel[i] + m1x;
            ia.vmean[n + i] = ia.vel[n + i] + m1y;
            ia.vmean[2 * n + i] = ia.vel[2 * n + i] + m1z;
            ia.sigma2[i] = T[4] / S0 - (m1x * m1x + m1y * m1y + m1z * m1z);
            ia.div[i] = T[5] * gs;
            ia.curl[i] = T[6] * gs;
            ia.curl[n + i] = T[7] * gs;
            ia.curl[2 * n + i] = T[8] * gs;
            ia.count[i] = count;
            pairs += (unsigned long long)count;
        }
        if (lane == 0) tests += (unsigned long long)staged * (unsigned long long)G;
    }
    pairs = warp_sum(pairs);
    if (lane == 0) {
        if (pairs) atomicAdd(&a.ds->pair_evals, pairs);
        if (tests) atomicAdd(&a.ds->pair_tests, tests);
    }
}

// Sorted velocity records from the caller's (3 x n) FP64 velocities; a non-finite component
// sets kBadVelocity.
template <bool kF64>
__global__ void k_gather_vel(const int32_t *__restrict__ idx, const double *__restrict__ vel, int64_t n,
                             void *__restrict__ vrec, DevState *ds)
{
    int bad = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx[p];
        const double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i];
        if (!(fabs(vx) <= DBL_MAX && fabs(vy) <= DBL_MAX && fabs(vz) <= DBL_MAX)) bad = 1;
        if (kF64) ((double4_32a *)vrec)[p] = make_double4_32a(vx, vy, vz, 0.0);
        else ((float4 *)vrec)[p] = make_float4((float)vx, (float)vy, (float)vz, 0.f);
    }
    if (bad) atomicOr(&ds->status, kBadVelocity);
}

template <bool kF64, int kKern>
cudaError_t launch_interact_t(const SolveArgs &a, const InteractArgs &ia, const int32_t *todo,
                              cudaStream_t st)
{
    constexpr int smem = kIWarps * interact_warp_bytes<kF64>();
    static_assert(smem <= 48 * 1024, "dynamic shared memory above 48 KB needs an opt-in per device");
    // a persistent grid: as many blocks as are resident on the current device
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interact<kF64, kKern>, kIThreads, smem);
    if (e != cudaSuccess) return e;
    k_interact<kF64, kKern><<<sms * (per_sm > 0 ? per_sm : 1), kIThreads, smem, st>>>(a, ia, todo);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interact(const SolveArgs &a, const InteractArgs &ia, const int32_t *todo, cudaStream_t st)
{
    const bool f64 = a.precision == 0;  // SPH_PREC_FP64
    if (f64) return a.kernel ? launch_interact_t<true, 1>(a, ia, todo, st) : launch_interact_t<true, 0>(a, ia, todo, st);
    return a.kernel ? launch_interact_t<false, 1>(a, ia, todo, st) : launch_interact_t<false, 0>(a, ia, todo, st);
}

cudaError_t launch_gather_vel(const SolveArgs &a, const double *vel, void *vrec, cudaStream_t st)
{
    int64_t b = (a.n + 255) / 256;
    if (b < 1) b = 1;
    const int grid = (int)(b < a.grid_cap ? b : a.grid_cap);
    if (a.precision == 0) k_gather_vel<true><<<grid, 256, 0, st>>>(a.idx, vel, a.n, vrec, a.ds);
    else k_gather_vel<false><<<grid, 256, 0, st>>>(a.idx, vel, a.n, vrec, a.ds);
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

}  // namespace sph
