// sph_kernels.cuh -- argument blocks and launchers of the sort and solve kernels.
#pragma once

#include "sph_common.cuh"

namespace sph {

// Buffers the sort stage reads and writes.
struct SortArgs {
    uint64_t *key[2];      // ping-pong key buffers
    int32_t *idx[2];       // ping-pong original-index buffers
    int32_t *hist;         // radix histograms
    int32_t *hist_off;     // their exclusive scan
    int32_t *scan_aux;     // scan scratch
    uint4 *pfix;           // sorted fixed-point positions + FP32 mass
    double4_32a *pdbl;         // sorted FP64 positions + mass
    int32_t *ctab;         // dense cell tables of all segments
    SegInfo *segs;         // segment descriptors (device)
    DevState *ds;
    KeyLayout kl;
    int grid_cap;          // upper bound on blocks per launch
    int table_extra;       // dense-table levels beyond one cell per particle (batch groups)
    double self_floor;     // N_w of a lone particle (32/3 M4, 1365/48 Wendland C6)
    int *launches;         // host-side launch counter
};

int64_t radix_hist_size(int64_t n_max);
// rec (nullable): caller-order fixed-point records for launch_gather_rec (FP32 sorts)
cudaError_t launch_keys_periodic(const SortArgs &a, int64_t n, const double *pos, const double *mass,
                                 const SegInfo &seg, const double box[3], cudaStream_t st,
                                 uint4 *rec = nullptr);
cudaError_t launch_group_setup(const SortArgs &a, int64_t n_groups, const int64_t *offsets,
                               const double *pos, int64_t n, const double *nngb, const double *tol,
                               int32_t *tsize, int32_t *toff, cudaStream_t st);
cudaError_t launch_keys_open(const SortArgs &a, int64_t n, const double *pos, const double *mass,
                             const int64_t *offsets, int64_t n_groups, cudaStream_t st,
                             uint4 *rec = nullptr);
cudaError_t launch_radix_sort(const SortArgs &a, int64_t n, int *which, cudaStream_t st);
cudaError_t launch_gather_periodic(const SortArgs &a, int64_t n, const double *pos,
                                   const double *mass, const int32_t *idx, const SegInfo &seg,
                                   cudaStream_t st);
cudaError_t launch_gather_open(const SortArgs &a, int64_t n, const double *pos, const double *mass,
                               const int32_t *idx, const uint64_t *key, cudaStream_t st);
// pfix[p] = rec[idx[p]]: the sorted fixed-point records without the FP64 ones
cudaError_t launch_gather_rec(const SortArgs &a, int64_t n, const int32_t *idx, const uint4 *rec,
                              cudaStream_t st);
cudaError_t launch_cell_table(const SortArgs &a, int64_t n, const uint64_t *key, cudaStream_t st);

// Buffers and state of the solve.
struct SolveArgs {
    // sorted particle data
    const uint4 *pfix;
    const double4_32a *pdbl;
    const uint64_t *key;
    const int32_t *idx;        // sorted position -> caller index
    const SegInfo *segs;
    const int32_t *ctab;
    KeyLayout kl;
    int64_t n;
    // iteration state (sorted order)
    double *h;                 // h of the next evaluation
    double *hlo, *hhi;         // brackets
    double *e_h;               // h of the last evaluation
    double *e_rho, *e_nw, *e_dnw;   // last evaluation (FP64 precision mode)
    int32_t *e_cnt;
    float *h32;                      // FP32 copy of h, read by the FP32 density kernel
    float *e_rho32, *e_nw32, *e_dnw32;  // last evaluation (FP32 precision mode)
    int32_t *todo[2];          // ping-pong todo lists (sorted positions)
    int32_t *flags;            // per-todo-entry scratch flags
    int32_t *items;            // work-item starts (indices into the todo list)
    int32_t *scan_aux;
    DevState *ds;
    int grid_cap;
    int density_grid;          // persistent blocks of the density kernels
    int gmax;                  // targets per work item (<= 32)
    int gmax_sparse;           // the same while the todo list is sparse (< 1/8 of the particles)
    int item_cap;              // 0: items follow the grouping level; else the coarsest octree
                               // cell (not coarser than that level) with <= item_cap todo targets
    int block_threads;         // threads per block of the density kernels (64, 128 or 256)
    int group_shift;           // items group targets sharing an octree cell of edge >= h / 2^shift
    int sparse_shift;          // the same while the todo list is sparse (< 1/8 of the particles)
    int cell_div;              // candidate cells have an edge >= (query extent) / cell_div
    int direct_pct;            // in-h percentage of the first tests above which the pair loop
                               // evaluates directly instead of queueing (101 = always queue)
    int precision;             // sph_precision
    int kernel;                // sph_kernel: 0 M4 cubic spline, 1 Wendland C6
    int free_first;            // 1: the first pass of a solve from one common h runs the
                               // branch-free FP32 pair loop (periodic FP32 direct solves)
    int cubic;                 // 1: equal fixed-point quanta in x, y, z (read by the kNN pass)
    int *launches;
    cudaEvent_t dens_ev[2];    // optional events recorded around the density launch
    // neighbour-set export of sampled targets (test aid; nb_out == nullptr: off).  The density
    // pass then also writes, for every target whose caller index i has nb_slot[i] = k >= 0, the
    // caller indices of its in-h neighbours to nb_out[k * nb_max ..] and their number to
    // nb_cnt[k] (counted in full; entries past nb_max are not written).
    const int32_t *nb_slot;
    int32_t *nb_out;
    int32_t *nb_cnt;
    int nb_max;
    // cached neighbour lists (lst == nullptr: off).  A neighbour search records, for each of its
    // targets p, the sorted positions of the particles within list_margin * h_p (at most
    // list_entries) in lst[p * list_entries ..], their number in lst_n[p] (-1: no list) and the
    // radius every h up to which the list serves in lst_r[p]; a later pass of the same solve whose
    // h stays within lst_r evaluates the list instead of searching (targets that search go
    // through todo_s)
    int32_t *lst;
    int32_t *lst_n;
    double *lst_r;
    int32_t *todo_s;
    int list_entries;
    float list_margin;         // > 1
};

// Buffers of the interaction pass (sph_interact.cu).
struct InteractArgs {
    const void *vrec;   // sorted velocities: float4 {vx, vy, vz, 0} (FP32 mode) or double4_32a
    const double *vel;  // caller velocities, 3 x n (x block, y block, z block)
    double *rho;        // outputs in caller order (vmean, curl: 3 x n)
    double *vmean;
    double *sigma2;
    double *div;
    double *curl;
    int32_t *count;
};

cudaError_t launch_solve_init(const SolveArgs &a, const double *h_in, int max_iter, cudaStream_t st);
// One evaluation pass over todo[cur]; when `update`, also the h update and the next todo
// list (todo[1 - cur]).
cudaError_t launch_pass(const SolveArgs &a, int cur, bool update, cudaStream_t st);
cudaError_t launch_set_loop(cudaGraphConditionalHandle handle, const DevState *ds, cudaStream_t st);
cudaError_t launch_scatter(const SolveArgs &a, double *h_out, double *rho_out, int32_t *count_out,
                           double *nw_out, double *dnw_out, cudaStream_t st);

// sph_density.cu
cudaError_t launch_density(const SolveArgs &a, const int32_t *todo, cudaStream_t st);
// evaluate the todo targets whose cached lists still cover their h; flags[t] = 1 for the others
cudaError_t launch_list_eval(const SolveArgs &a, const int32_t *todo, cudaStream_t st);
// resident blocks per SM of the density kernel of this precision / mode at this block size
int density_blocks_per_sm(int precision, int direct_pct, int block_threads = 256);
// k-nearest-neighbour pass over todo (one warp per target): selects h for targets whose
// search radius holds K..knn_capacity candidates, adapts the radius of the others
cudaError_t launch_knn(const SolveArgs &a, const int32_t *todo, int k, cudaStream_t st);
int knn_capacity(int precision);
// sph_solve.cu: one kNN pass (selection + next todo list), and the switch to one density
// evaluation of every particle at its selected h
cudaError_t launch_knn_pass(const SolveArgs &a, int cur, int k, cudaStream_t st);
cudaError_t launch_knn_finish(const SolveArgs &a, cudaStream_t st);
// starting radii of the kNN passes (entries <= 0 are estimated from the cell tables)
cudaError_t launch_knn_init(const SolveArgs &a, const double *h_in, int max_iter, int k, cudaStream_t st);
// sph_interact.cu: the interaction kernel over the items of todo, and the sorted velocity
// records (status bit kBadVelocity for a non-finite component)
cudaError_t launch_interact(const SolveArgs &a, const InteractArgs &ia, const int32_t *todo, cudaStream_t st);
cudaError_t launch_gather_vel(const SolveArgs &a, const double *vel, void *vrec, cudaStream_t st);
// sph_solve.cu: one interaction pass over every particle (after launch_solve_init with one pass)
cudaError_t launch_interact_pass(const SolveArgs &a, const InteractArgs &ia, cudaStream_t st);
// neighbour export set-up: nb_slot (caller order, n entries) = -1 except nb_slot[sample[k]] = k;
// counts zeroed; an index outside [0, n) or repeated sets kBadSample in the status word
cudaError_t launch_nb_setup(const SolveArgs &a, int32_t *nb_slot, const int64_t *sample, int64_t n_sample,
                            int32_t *nb_cnt, cudaStream_t st);

}  // namespace sph
