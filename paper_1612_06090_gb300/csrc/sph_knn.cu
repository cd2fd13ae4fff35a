// sph_knn.cu -- k-nearest-neighbour smoothing lengths (Sec. IV-D): one warp per target streams
// the candidates inside the target's search radius, keeps their squared distances in a buffer
// cut back to its K nearest when full, and selects the K-th with a warp radix select.
#include <climits>
#include <cstring>
#include <type_traits>

#include "sph_items.cuh"
#include "sph_kernels.cuh"

namespace sph {

namespace {

// ---- k-nearest-neighbour smoothing length (Sec. IV-D) --------------------------------------
//
// The Subfind form of the density loop orders each particle's neighbour list by distance and
// keeps the K nearest.  Here one warp owns one target: it streams the candidates inside the
// target's current search radius H (the same culled cell stream as the density pass) and keeps
// their squared distances in a per-warp buffer, cut back to its K nearest whenever it would
// overflow.  With at least K candidates inside H the K-th smallest is selected with a warp radix
// select (8-bit digits on the IEEE bit patterns, which order non-negative floats); h = sqrt of
// it.  With fewer, H grows and the target returns in the next pass.
// FP32: squared distances of the FP32 offsets, as in the FP32 density pairs.  FP64: formed
// from the FP64 positions exactly as the FP64 pairs (and the oracle) form them.

constexpr int kKnnWarps = 8;
constexpr int kKnnThreads = 32 * kKnnWarps;
constexpr int kKnnCap = 896;   // buffered candidates per warp (>= SPH_KNN_MAX_K + 256)
constexpr int kKnnLoads = 4;   // independent candidate loads per lane per stream round

template <bool kF64>
__host__ __device__ constexpr int knn_cap() { return kKnnCap; }
template <bool kF64>
__host__ __device__ constexpr int knn_buf_bytes() { return kKnnCap * (kF64 ? 8 + 4 : 4 + 4); }
template <bool kF64>
__host__ __device__ constexpr int knn_warp_bytes() { return knn_buf_bytes<kF64>() + 256 * 4 + 2 * kMaxCells * 4; }

// K-th smallest (1-based) of the c keys; every round keeps the keys that agree with the digits
// chosen so far and histograms their next digit.
template <typename U>
__device__ __forceinline__ U radix_select(const U *__restrict__ keys, int c, int K, int *hist)
{
    const int lane = lane_id();
    U prefix = 0, mask = 0;
    int kk = K;
#pragma unroll 1
    for (int shift = 8 * (int)sizeof(U) - 8; shift >= 0; shift -= 8) {
        for (int b = lane; b < 256; b += 32) hist[b] = 0;
        __syncwarp();
        for (int i = lane; i < c; i += 32) {
            const U v = keys[i];
            if ((v & mask) == prefix) atomicAdd(&hist[(int)((v >> shift) & 0xff)], 1);
        }
        __syncwarp();
        int loc[8];
        int sum = 0;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            loc[q] = hist[8 * lane + q];
            sum += loc[q];
        }
        const int incl = warp_inclusive_scan(sum);
        const int excl = incl - sum;
        const bool mine = excl < kk && kk <= incl;
        int bin = 0, below = 0;
        if (mine) {
            int acc = excl;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                if (bin == 0 && below == 0 && acc + loc[q] >= kk && acc < kk) {
                    bin = 8 * lane + q;
                    below = acc;
                }
                acc += loc[q];
            }
        }
        const int src = __ffs(__ballot_sync(kFull, mine)) - 1;
        bin = __shfl_sync(kFull, bin, src);
        below = __shfl_sync(kFull, below, src);
        kk -= below;
        prefix |= (U)bin << shift;
        mask |= (U)0xff << shift;
        __syncwarp();
    }
    return prefix;
}

// rho, N_w and the count at h over the buffered candidates (the target's own entry included),
// in the precision of the pass (FP32 entries are squared distances in units of u2).  FP64: the oracle's pair terms; FP32: single-precision terms and
// sums (at most K - 1 + ties terms per target).
template <bool kF64, typename T>
__device__ void knn_density(const SolveArgs &a, int p, double h, const T *__restrict__ buf,
                            const int *__restrict__ bidx, int c, float u2)
{
    const int lane = lane_id();
    const bool c6 = a.kernel != 0;
    if (kF64) {
        const double h2 = __dmul_rn(h, h);
        double smw = 0.0, sw = 0.0;
        int cnt = 0;
        for (int i = lane; i < c; i += 32) {
            const double r2 = (double)buf[i];
            if (r2 < h2) {
                const double q = __ddiv_rn(__dsqrt_rn(r2), h);
                double w;
                if (c6) {
                    const double u = __dsub_rn(1.0, q), u2 = __dmul_rn(u, u), u4 = __dmul_rn(u2, u2);
                    const double poly = __dadd_rn(__dadd_rn(__dadd_rn(1.0, __dmul_rn(8.0, q)),
                                                            __dmul_rn(25.0, __dmul_rn(q, q))),
                                                  __dmul_rn(32.0, __dmul_rn(__dmul_rn(q, q), q)));
                    w = __dmul_rn(__dmul_rn(u4, u4), poly);
                } else if (q <= 0.5) {
                    w = __dadd_rn(1.0, __dmul_rn(__dmul_rn(q, q), __dsub_rn(__dmul_rn(6.0, q), 6.0)));
                } else {
                    const double u = __dsub_rn(1.0, q);
                    w = __dmul_rn(2.0, __dmul_rn(__dmul_rn(u, u), u));
                }
                smw = __dadd_rn(smw, __dmul_rn(a.pdbl[bidx[i]].w, w));
                sw = __dadd_rn(sw, w);
                cnt++;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            smw += __shfl_xor_sync(kFull, smw, o);
            sw += __shfl_xor_sync(kFull, sw, o);
        }
        cnt = __reduce_add_sync(kFull, cnt);
        if (lane == 0) {
            const double kPi = 3.14159265358979323846;
            a.e_h[p] = h;
            a.e_rho[p] = smw * (c6 ? 1365.0 / (64.0 * kPi * h * h * h) : 8.0 / (kPi * h * h * h));
            a.e_nw[p] = (c6 ? 1365.0 / 48.0 : 32.0 / 3.0) * sw;
            a.e_cnt[p] = cnt;
        }
    } else {
        const float hf = (float)h, h2 = hf * hf, hinv = 1.0f / hf;
        float smw = 0.f, sw = 0.f;
        int cnt = 0;
        for (int i = lane; i < c; i += 32) {
            const float r2 = (float)buf[i] * u2;  // FP32 entries are in units of u2
            if (r2 < h2) {
                const float q = sqrtf(r2) * hinv;
                float w;
                if (c6) {
                    const float u = fmaxf(1.f - q, 0.f), u2 = u * u, u4 = u2 * u2;
                    w = u4 * u4 * fmaf(q, fmaf(q, fmaf(q, 32.f, 25.f), 8.f), 1.f);
                } else if (q <= 0.5f) {
                    w = fmaf(q * q, fmaf(6.f, q, -6.f), 1.f);
                } else {
                    const float u = fmaxf(1.f - q, 0.f);
                    w = 2.f * u * u * u;
                }
                smw = fmaf(__uint_as_float(a.pfix[bidx[i]].w), w, smw);
                sw += w;
                cnt++;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            smw += __shfl_xor_sync(kFull, smw, o);
            sw += __shfl_xor_sync(kFull, sw, o);
        }
        cnt = __reduce_add_sync(kFull, cnt);
        if (lane == 0) {
            const float kPif = 3.14159265f;
            a.e_h[p] = h;
            a.e_rho32[p] = smw * (c6 ? 1365.0f / (64.0f * kPif) : 8.0f / kPif) * (hinv * hinv * hinv);
            a.e_nw32[p] = (c6 ? 1365.0f / 48.0f : 32.0f / 3.0f) * sw;
            a.e_cnt[p] = cnt;
        }
    }
}

// kCubic: the three fixed-point quanta are equal (a cubic box), so squared distances are formed
// in units of q^2 from the integer offsets directly and converted once per target.
template <bool kF64, bool kCubic>
__global__ void __launch_bounds__(kKnnThreads, kF64 ? 2 : 3)
    k_knn(SolveArgs a, const int32_t *__restrict__ todo, int K)
{
    using T = typename std::conditional<kF64, double, float>::type;
    using U = typename std::conditional<kF64, unsigned long long, unsigned>::type;
    constexpr int cap = knn_cap<kF64>();
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wb = smem + (size_t)warp * knn_warp_bytes<kF64>();
    T *buf = (T *)wb;                          // squared distances
    int *bidx = (int *)(wb + kKnnCap * sizeof(T));  // their candidates' sorted positions
    int *hist = (int *)(wb + knn_buf_bytes<kF64>());
    int *cpre = hist + 256;
    int *cbeg = cpre + kMaxCells;
    const int n_todo = a.ds->pass_count;
    const int pass = a.ds->pass;
    int exceeded = 0;
    unsigned long long tests = 0, listed = 0;

    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&a.ds->item_head, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_todo) break;
        const int p = todo[t];
        const double H = a.h[p];
        const uint4 P = a.pfix[p];
        const int g = a.kl.seg_bits > 0 ? (int)(a.key[p] >> (3 * a.kl.lmax)) : 0;
        const SegInfo &S = a.segs[g];
        const float Hf = (float)H;
        ItemGeom G3;
        int rel[3];
        // the box only needs to contain the ball of radius H, so the FP32 radius is enlarged
        item_setup(S, a.kl, a.cell_div, true, P, Hf * (1.0f + 1.0f / 1048576.0f), G3, rel);
        const float qf[3] = {(float)S.q[0], (float)S.q[1], (float)S.q[2]};
        const float qm = fmaxf(qf[0], fmaxf(qf[1], qf[2]));
        const float Rm = Hf * (1.0f + 1e-5f) + 8.0f * qm;
        const float ball2 = Rm * Rm;
        const int ncell = G3.nc[0] * G3.nc[1] * G3.nc[2];
        if (ncell > kMaxCells) {  // cannot happen by construction; report, never overrun
            if (lane == 0) atomicOr(&a.ds->status, 8);
            continue;
        }
        long long rr[2];
        {
            const float cc[3] = {0.f, 0.f, 0.f};
            item_ranges(G3, g, S, a.kl, a.ctab, a.key, ncell, cc, ball2, qf, rr);
        }
        // FP32 distances are in units of u2 = q^2 when the box is cubic, else in box units
        const float uq = kCubic ? qf[0] : 1.0f;
        const float u2 = uq * uq;
        const float Hu = Hf / uq;
        const float H2f = Hu * Hu;
        const float ball2u = kCubic ? ball2 / u2 : ball2;
        const double H2 = __dmul_rn(H, H);
        double4_32a ti = make_double4_32a(0, 0, 0, 0);
        if (kF64) ti = a.pdbl[p];

        int total;
        {
            const int b0 = (int)(rr[0] & 0xffffffffll), n0 = (int)(rr[0] >> 32) - b0;
            const int b1 = (int)(rr[1] & 0xffffffffll), n1 = (int)(rr[1] >> 32) - b1;
            const int i0 = warp_inclusive_scan(n0), i1 = warp_inclusive_scan(n1);
            const int tot0 = __shfl_sync(kFull, i0, 31);
            total = tot0 + __shfl_sync(kFull, i1, 31);
            __syncwarp();
            cpre[lane] = i0 - n0;
            cbeg[lane] = b0 - (i0 - n0);  // index offset: particle = position + offset
            cpre[lane + 32] = tot0 + i1 - n1;
            cbeg[lane + 32] = b1 - (tot0 + i1 - n1);
            __syncwarp();
        }
        int cc = 0, coff = cbeg[0], cnxt = cpre[1];
        // The buffer holds candidates inside H.  When it would overflow it is cut to the
        // entries at or below its K-th smallest value tau; from then on only candidates at or
        // below tau enter (tau only falls, so every value below the final tau stays, and the
        // K-th smallest of the buffer at the end is the K-th smallest inside H).  Until the
        // first cut the buffer holds every candidate inside H, so c is their count.
        int c = 0;     // entries in the buffer
        bool cut = false, stuck = false;
        T tau = 0;
        for (int base = 0; base < total; base += 32 * kKnnLoads) {
          // the round's loads are all issued before any is used
          int jj[kKnnLoads];
          uint4 PP[kKnnLoads];
#pragma unroll
          for (int u = 0; u < kKnnLoads; u++) {
            const int f = base + 32 * u + lane;
            if (f < total && cnxt <= f) {
                // positions only grow: step to the cell holding f (empty cells are passed over)
                int ci = cc;
                while (ci + 1 < kMaxCells && cpre[ci + 1] <= f) ci++;
                cc = ci;
                coff = cbeg[ci];
                cnxt = ci + 1 < kMaxCells ? cpre[ci + 1] : INT_MAX;
            }
            jj[u] = f < total ? f + coff : -1;
            PP[u] = make_uint4(0, 0, 0, 0);
            if (jj[u] >= 0) PP[u] = a.pfix[jj[u]];
          }
#pragma unroll
          for (int u = 0; u < kKnnLoads; u++) {
            const int j = jj[u];
            bool in = false;
            T r2 = 0;
            if (j >= 0) {
                // one target: its offsets are wrapped minimum images, and a candidate outside
                // the query box also fails the radius test, so no box test is needed
                const uint4 Pj = PP[u];
                const int rj[3] = {(int32_t)(Pj.x - G3.X0[0]), (int32_t)(Pj.y - G3.X0[1]),
                                   (int32_t)(Pj.z - G3.X0[2])};
                {
                    const float fx = kCubic ? (float)rj[0] : (float)rj[0] * qf[0];
                    const float fy = kCubic ? (float)rj[1] : (float)rj[1] * qf[1];
                    const float fz = kCubic ? (float)rj[2] : (float)rj[2] * qf[2];
                    const float r2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
                    if (kF64) {
                        if (r2f <= ball2u) {
                            const double4_32a cj = a.pdbl[j];
                            double dx = __dsub_rn(cj.x, ti.x);
                            double dy = __dsub_rn(cj.y, ti.y);
                            double dz = __dsub_rn(cj.z, ti.z);
                            if (S.periodic) {
                                dx = min_image64(dx, S.box[0]);
                                dy = min_image64(dy, S.box[1]);
                                dz = min_image64(dz, S.box[2]);
                            }
                            const double d2 =
                                __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                            r2 = (T)d2;
                            in = d2 < H2;
                        }
                    } else {
                        r2 = (T)r2f;
                        in = r2f < H2f;
                    }
                }
            }
            bool keep = in && (!cut || r2 <= tau);
            unsigned m = __ballot_sync(kFull, keep);
            if (c + __popc(m) > cap && !stuck) {
                const U kth = radix_select<U>((const U *)buf, c, K, hist);
                memcpy(&tau, &kth, sizeof(T));
                cut = true;
                int nc = 0;
                for (int i0 = 0; i0 < c; i0 += 32) {
                    const int i = i0 + lane;
                    T v = 0;
                    int vj = 0;
                    bool kp = false;
                    if (i < c) {
                        v = buf[i];
                        vj = bidx[i];
                        kp = v <= tau;
                    }
                    __syncwarp();  // the round's reads come before any of its writes
                    const unsigned km = __ballot_sync(kFull, kp);
                    if (kp) {
                        buf[nc + __popc(km & lanemask_lt())] = v;
                        bidx[nc + __popc(km & lanemask_lt())] = vj;
                    }
                    nc += __popc(km);
                    __syncwarp();
                }
                c = nc;
                // more than cap - 32 entries equal tau: no room can be made (handled below)
                stuck = c + 32 > cap;
                keep = in && r2 <= tau;
                m = __ballot_sync(kFull, keep);
            }
            if (!stuck) {
                if (keep) {
                    const int slot = c + __popc(m & lanemask_lt());
                    buf[slot] = r2;
                    bidx[slot] = j;
                }
                c += __popc(m);
            }
          }
        }
        tests += (unsigned long long)total;
        listed += (unsigned long long)c;
        __syncwarp();

        int alive = 0;
        if ((cut || c >= K) && !stuck) {
            const U key = radix_select<U>((const U *)buf, c, K, hist);
            T r2k;
            memcpy(&r2k, &key, sizeof(T));
            const double h = kF64 ? __dsqrt_rn((double)r2k) : sqrt((double)r2k) * (double)uq;
            if (S.periodic && h >= S.half_box) {
                exceeded++;
                if (lane == 0) a.e_h[p] = H;
            } else {
                // Eq. 1 at h from the buffer: every particle with r < h is in it (all entries
                // at or below tau >= r_K^2 were kept)
                knn_density<kF64>(a, p, h, buf, bidx, c, u2);
            }
        } else {
            // bracket: lo holds fewer than K candidates, hi a radius where the buffer could not
            // be cut.  Growing, the count is taken to scale as H^3 and H aims at 2K candidates;
            // with both sides known the bracket is halved geometrically (the count is monotone
            // in H, so this ends even where density changes steeply)
            double lo = a.hlo[p], hi = a.hhi[p];
            if (!cut) lo = H;  // fewer than K inside H
            else hi = H;  // stuck: thousands of equal distances inside H
            double hn;
            if (lo > 0.0 && hi < HUGE_VAL) {
                hn = sqrt(lo * hi);
            } else if (!cut) {
                hn = H * fmin(fmax(cbrt(2.0 * K / (double)(c > 0 ? c : 1)), 1.05), 4.0);
            } else {
                hn = H * 0.5;
            }
            if (lane == 0) {
                a.hlo[p] = lo;
                a.hhi[p] = hi;
            }
            if (S.periodic && hn >= S.half_box) {
                if (H >= S.half_box * 0.9999) {
                    exceeded++;  // fewer than K particles within the largest legal radius
                    hn = H;
                } else {
                    hn = S.half_box * 0.99999;
                    alive = 1;
                }
            } else {
                alive = 1;
            }
            if (lane == 0) {
                a.h[p] = hn;
                a.h32[p] = (float)hn;
                a.e_h[p] = hn;
            }
        }
        if (lane == 0) a.flags[t] = alive;
    }
    if (lane == 0) {
        if (exceeded) atomicAdd(&a.ds->exceeded, exceeded);
        if (tests) atomicAdd(&a.ds->pair_tests, tests);
        if (listed) {
            atomicAdd(&a.ds->pair_evals, listed);
            if (pass < kMaxPasses) atomicAdd(&a.ds->pairs_per_pass[pass], listed);
        }
    }
}

}  // namespace

template <bool kF64, bool kCubic>
int knn_blocks_per_sm()
{
    const int bytes = kKnnWarps * knn_warp_bytes<kF64>();
    cudaFuncSetAttribute(k_knn<kF64, kCubic>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_knn<kF64, kCubic>, kKnnThreads, bytes);
    return b > 0 ? b : 1;
}

template <bool kF64, bool kCubic>
void knn_launch(const SolveArgs &a, const int32_t *todo, int k, int sms, cudaStream_t st)
{
    k_knn<kF64, kCubic><<<sms * knn_blocks_per_sm<kF64, kCubic>(), kKnnThreads,
                          kKnnWarps * knn_warp_bytes<kF64>(), st>>>(a, todo, k);
}

int knn_capacity(int precision) { return precision == 0 ? knn_cap<true>() : knn_cap<false>(); }

cudaError_t launch_knn(const SolveArgs &a, const int32_t *todo, int k, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (a.precision == 0) {
        if (a.cubic) knn_launch<true, true>(a, todo, k, sms, st);
        else knn_launch<true, false>(a, todo, k, sms, st);
    } else {
        if (a.cubic) knn_launch<false, true>(a, todo, k, sms, st);
        else knn_launch<false, false>(a, todo, k, sms, st);
    }
    if (a.launches) *a.launches += 1;
    return cudaGetLastError();
}

}  // namespace sph
