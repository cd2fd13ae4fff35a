// sph_common.cuh -- types and device helpers shared by the CUDA translation units.
//
// Particle representation on the device (sorted order):
//   pfix[p] = {X, Y, Z, bits(m)}: 32-bit fixed-point coordinates and the FP32 mass.
//     Periodic: X = floor(x / L_x * 2^32) in [0, 2^32); the wrapped int32 difference of
//     two coordinates is the minimum-image separation in units of q_x = L_x / 2^32.
//     Open (batch groups): X = floor((x - o_x) / q) in [0, 2^31) with one cubic quantum
//     q = extent / 2^31 per group; int32 differences never wrap.
//   pdbl[p] = {x, y, z, m} in FP64 (the FP64 precision mode reads these).
// Keys: (segment << 3*lmax) | Morton(X >> (B - lmax), ..) with B = 32 (periodic) or 31
// (open).  A cell of
// level l (l <= lmax) is the set of keys sharing the top seg_bits + 3*l bits, which is a
// contiguous range of the sorted arrays.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sph {

constexpr int kWarp = 32;
constexpr int kMaxPasses = 64;
constexpr unsigned kFull = 0xffffffffu;

// Per-segment (one periodic system, or one batch group) geometry and targets.
struct SegInfo {
    double q[3];       // length of one fixed-point unit per dimension
    double inv_q[3];   // 1 / q
    double origin[3];  // open boundaries: coordinate of X = 0
    double box[3];     // periodic box lengths (exactly q * 2^32)
    double nngb;       // target weighted count
    double tol;        // band half-width
    double half_box;   // periodic: min(box) / 2, the h limit; open: +inf
    int32_t periodic;  // 1: 32-bit wrapped coordinates; 0: 31-bit open coordinates
    int32_t level_c;   // level of the dense cell table
    int32_t tab_off;   // offset of the segment's table in the table buffer
    int32_t start;     // sorted range [start, end)
    int32_t end;
    int32_t pad;
};

// Layout of the sort key.
struct KeyLayout {
    int32_t lmax;        // Morton levels in the key (bits per dimension)
    int32_t seg_bits;    // bits above the Morton part holding the segment id
    int32_t key_bits;    // seg_bits + 3 * lmax
    int32_t coord_bits;  // 32 (periodic, wrapped) or 31 (open); the level-l cell of a
                         // coordinate X is X >> (coord_bits - l)
};

// Counters and flags that live in device memory (one struct per context).
struct DevState {
    int32_t todo_count;        // entries in the current todo list
    int32_t todo_next;         // entries written to the next todo list
    int32_t n_items;           // work items in the current pass
    int32_t item_head;         // work-queue head (persistent kernels pop from here)
    int32_t status;            // bit flags of device-detected input errors
    int32_t exceeded;          // particles stopped by the box limit
    int32_t pass;              // passes completed
    int32_t max_iter;          // pass limit
    int32_t loop_flag;         // 1 while another pass is needed (device-side loop)
    int32_t pass_count;        // entries this pass evaluates (0: the pass is skipped)
    int32_t sort_status;       // input errors found by the sort (kept across solves)
    int32_t h_varies;          // some starting h differs from particle 0's (set by the solve init)
    int32_t free_now;          // this pass runs the branch-free FP32 pair loop
    int32_t dens_count;        // entries of this pass that the neighbour search evaluates (all of
                               // them, or those without a usable cached neighbour list)
    unsigned long long pair_evals;  // in-h pairs accumulated over the solve
    unsigned long long pair_tests;  // candidate-target distance tests (work done, not counted
                                    // as algorithmic work)
    unsigned long long list_evals;  // target evaluations served by cached neighbour lists
    int32_t todo_per_pass[kMaxPasses];
    unsigned long long pairs_per_pass[kMaxPasses];
};

enum DevStatusBits : int32_t {
    kBadPosition = 1,   // NaN/Inf coordinate, or outside [0, box) when periodic
    kBadMass = 2,       // mass not finite or <= 0
    kBadH = 4,          // h not finite, <= 0, or >= min(box)/2 when periodic
    kBadSample = 16,    // neighbour export: a sample index outside [0, n) or repeated
    kBadVelocity = 32,  // interaction pass: a velocity component not finite
};

// ---------------------------------------------------------------------------------------
// Morton interleave of three 21-bit values: bit b of x goes to bit 3b, y to 3b+1, z to 3b+2.
// ---------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t spread_bits3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__host__ __device__ __forceinline__ uint64_t morton3(uint32_t cx, uint32_t cy, uint32_t cz)
{
    return spread_bits3(cx) | (spread_bits3(cy) << 1) | (spread_bits3(cz) << 2);
}

// ---------------------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Inclusive scan across the warp.
__device__ __forceinline__ int warp_inclusive_scan(int v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Host-side error checking helper for the orchestration code.
#define SPH_CUDA_TRY(expr)                                                                   \
    do {                                                                                     \
        cudaError_t err__ = (expr);                                                          \
        if (err__ != cudaSuccess) return err__;                                              \
    } while (0)

// ---------------------------------------------------------------------------------------
// Launchers implemented in the .cu files (all asynchronous on `st`).
// ---------------------------------------------------------------------------------------

// sph_scan.cu: exclusive prefix sum of n int32 values (n read from n_dev when non-null,
// else n_host).  total_dev (optional) receives the sum.  aux needs scan_aux_size(n_max).
int64_t scan_aux_size(int64_t n_max);
cudaError_t scan_exclusive(const int32_t *in, int32_t *out, int64_t n_host, const int32_t *n_dev,
                           int32_t *total_dev, int32_t *aux, int grid_cap, cudaStream_t st,
                           int *launches);
// Stable compaction: out[k] = src[i] (i itself when src is null) for the i with
// flags[i] != 0, in order; the count goes to count_dev.  pos is unused (may be null).
cudaError_t compact_i32(const int32_t *flags, const int32_t *src, int32_t *out, int32_t *pos,
                        int64_t n_host, const int32_t *n_dev, int32_t *count_dev, int32_t *aux,
                        int grid_cap, cudaStream_t st, int *launches);

}  // namespace sph
