// sph_scan.cu -- device-wide exclusive prefix sums and stable stream compaction.
//
// Three launches with fixed grids (so they can sit in a CUDA graph while the element
// count lives in device memory): per-tile sums, one-block scan of the tile sums, and a
// per-tile scan that adds the tile offset.  The compaction variant writes the selected
// source values in their original order (the todo list keeps its spatial order, which
// the work-item grouping relies on).
#include "sph_common.cuh"

namespace sph {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;
constexpr int kAuxThreads = 1024;

__device__ __forceinline__ int64_t count_of(int64_t n_host, const int32_t *n_dev)
{
    return n_dev ? (int64_t)(*n_dev) : n_host;
}

// Exclusive scan of one value per thread across the block; returns the block total.
__device__ int block_exclusive_scan(int v, int &excl, int *warp_tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int inc = warp_inclusive_scan(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int t = lane < nwarps ? warp_tot[lane] : 0;
        int ti = warp_inclusive_scan(t);
        if (lane < nwarps) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == 31) warp_tot[32] = ti;           // block total
    }
    __syncthreads();
    excl = warp_tot[warp] + inc - v;
    int total = warp_tot[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kThreads) k_tile_sums(const int32_t *__restrict__ in,
                                                        int64_t n_host, const int32_t *n_dev,
                                                        int32_t *__restrict__ aux)
{
    __shared__ int warp_tot[33];
    const int64_t n = count_of(n_host, n_dev);
    const int64_t tiles = (n + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t base = t * kTile;
        int s = 0;
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
            if (i < n) s += in[i];
        }
        int excl;
        int tot = block_exclusive_scan(s, excl, warp_tot);
        if (threadIdx.x == 0) aux[t] = tot;
    }
}

__global__ void __launch_bounds__(kAuxThreads) k_scan_aux(int32_t *__restrict__ aux, int64_t n_host,
                                                          const int32_t *n_dev,
                                                          int32_t *total_dev)
{
    __shared__ int warp_tot[33];
    const int64_t n = count_of(n_host, n_dev);
    const int64_t tiles = (n + kTile - 1) / kTile;
    int carry = 0;
    for (int64_t b = 0; b < tiles; b += kAuxThreads) {
        int64_t i = b + threadIdx.x;
        int v = i < tiles ? aux[i] : 0;
        int excl;
        int tot = block_exclusive_scan(v, excl, warp_tot);
        if (i < tiles) aux[i] = carry + excl;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        aux[tiles] = carry;
        if (total_dev) *total_dev = carry;
    }
}

// kCompact = false: out[i] = exclusive prefix of in at i.
// kCompact = true : out[prefix(i)] = src[i] (or i when src is null) wherever in[i] != 0
//                   (in holds 0/1 flags).
template <bool kCompact>
__global__ void __launch_bounds__(kThreads) k_tile_scan(const int32_t *__restrict__ in,
                                                        const int32_t *__restrict__ src,
                                                        int32_t *__restrict__ out, int64_t n_host,
                                                        const int32_t *n_dev,
                                                        const int32_t *__restrict__ aux)
{
    __shared__ int tile[kTile];
    __shared__ int warp_tot[33];
    const int64_t n = count_of(n_host, n_dev);
    const int64_t tiles = (n + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t base = t * kTile;
        // striped, coalesced load into shared memory
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            int j = k * kThreads + threadIdx.x;
            int64_t i = base + j;
            tile[j] = i < n ? in[i] : 0;
        }
        __syncthreads();
        // each thread scans kItems consecutive values
        int v[kItems];
        int s = 0;
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            v[k] = tile[threadIdx.x * kItems + k];
            s += v[k];
        }
        int excl;
        block_exclusive_scan(s, excl, warp_tot);
        const int off = aux[t];
        int run = off + excl;
        if (kCompact) {
#pragma unroll
            for (int k = 0; k < kItems; k++) {
                int64_t i = base + threadIdx.x * kItems + k;
                if (v[k] != 0 && i < n) out[run] = src ? src[i] : (int32_t)i;
                run += v[k];
            }
            __syncthreads();
        } else {
#pragma unroll
            for (int k = 0; k < kItems; k++) {
                tile[threadIdx.x * kItems + k] = run;
                run += v[k];
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kItems; k++) {
                int j = k * kThreads + threadIdx.x;
                int64_t i = base + j;
                if (i < n) out[i] = tile[j];
            }
            __syncthreads();
        }
    }
}

int grid_for(int64_t n_max, int grid_cap)
{
    int64_t tiles = (n_max + kTile - 1) / kTile;
    if (tiles < 1) tiles = 1;
    return (int)(tiles < grid_cap ? tiles : grid_cap);
}

}  // namespace

int64_t scan_aux_size(int64_t n_max) { return (n_max + kTile - 1) / kTile + 2; }

cudaError_t scan_exclusive(const int32_t *in, int32_t *out, int64_t n_host, const int32_t *n_dev,
                           int32_t *total_dev, int32_t *aux, int grid_cap, cudaStream_t st,
                           int *launches)
{
    const int grid = grid_for(n_host, grid_cap);
    k_tile_sums<<<grid, kThreads, 0, st>>>(in, n_host, n_dev, aux);
    k_scan_aux<<<1, kAuxThreads, 0, st>>>(aux, n_host, n_dev, total_dev);
    k_tile_scan<false><<<grid, kThreads, 0, st>>>(in, nullptr, out, n_host, n_dev, aux);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

cudaError_t compact_i32(const int32_t *flags, const int32_t *src, int32_t *out, int32_t *pos,
                        int64_t n_host, const int32_t *n_dev, int32_t *count_dev, int32_t *aux,
                        int grid_cap, cudaStream_t st, int *launches)
{
    (void)pos;
    const int grid = grid_for(n_host, grid_cap);
    k_tile_sums<<<grid, kThreads, 0, st>>>(flags, n_host, n_dev, aux);
    k_scan_aux<<<1, kAuxThreads, 0, st>>>(aux, n_host, n_dev, count_dev);
    k_tile_scan<true><<<grid, kThreads, 0, st>>>(flags, src, out, n_host, n_dev, aux);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace sph
