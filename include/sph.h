/*
 * sph.h -- C ABI of the GB300 SPH density / smoothing-length solver.
 *
 * The library computes, for every particle i, the SPH density by kernel interpolation
 * (Baruffa et al., arXiv:1612.06090, Eq. 1, read in gather form):
 *     rho_i = sum_{j : r_ij < h_i} m_j W(r_ij, h_i),
 * with the M4 cubic-spline kernel W(r, h) = 8/(pi h^3) w(r/h), the self pair included,
 * together with the weighted neighbour count N_w = (4 pi / 3) h^3 sum_j W(r_ij, h), its
 * derivative dN_w/dh and the integer count n_i = #{j : r_ij < h_i}.  It adjusts each h_i
 * (Newton step with a bisection fallback) until |N_w - Nngb| <= tol, recomputing only
 * the particles still off target on every pass (Sec. IV-A, Listings 2 and 3:
 * mark_for_recomputation over a "todo" list with dynamic scheduling).  The paper states
 * no update rule; the one implemented is:
 *     converged iff |N_w - Nngb| <= tol; bracket: N_w < Nngb -> h_lo = h, else h_hi = h;
 *     Newton h' = h - (N_w - Nngb)/N_w' taken iff N_w' > 0, h_lo < h' < h_hi and
 *     h/2 <= h' <= 2h; otherwise (h_lo + h_hi)/2 when both bounds are set, h * 2^(1/3)
 *     when only h_lo is set, h / 2^(1/3) when only h_hi is set.  The h update and the
 *     convergence test always run in IEEE FP64.
 *
 * Memory and streams.  Every pointer argument named *_dev is DEVICE memory owned by the
 * caller, valid for the duration of the call and ordered on the context's stream.  A
 * context owns all scratch memory; it allocates it once, in sph_create, for `capacity`
 * particles, and never allocates afterwards.  One context per stream; a context is not
 * thread-safe.  Results are returned in the caller's particle order.
 *
 * Errors.  Every call returns an sph_status; nothing is thrown and nothing exits.
 * Argument errors are detected on the host before any device work is queued.  Errors
 * found on the device (non-finite or out-of-box positions, non-positive h) come back
 * through a device status word as SPH_ERR_DEVICE_STATUS.  sph_last_error() gives a
 * one-line description of the last failure on a context.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_ERR_INVALID_ARG = 1,    /* a bad argument, detected on the host                  */
    SPH_ERR_CUDA = 2,           /* a CUDA runtime call failed (no device, launch error)   */
    SPH_ERR_OOM = 3,            /* n or the group count exceeds the context's capacity    */
    SPH_ERR_NOT_SORTED = 4,     /* sph_density_solve/_eval before a successful sph_sort   */
    SPH_ERR_H_EXCEEDS_BOX = 5,  /* periodic: some h had to reach min(box)/2               */
    SPH_ERR_NOT_CONVERGED = 6,  /* max_iter passes ran out for some particles             */
    SPH_ERR_DEVICE_STATUS = 7,  /* the device flagged bad input (NaN/Inf/out-of-box)      */
    SPH_ERR_UNSUPPORTED = 8     /* a valid option this library does not implement        */
} sph_status;

typedef enum { SPH_KERNEL_M4 = 0, SPH_KERNEL_WENDLAND_C6 = 1 } sph_kernel;

/* FP64: every pair in FP64, exactly as the FP64 reference formulae are written.
 * FP32_KAHAN: pair distances and kernel weights in FP32 on offsets formed from
 * 32-bit fixed-point coordinates, sums compensated (Kahan), h update in FP64. */
typedef enum { SPH_PREC_FP64 = 0, SPH_PREC_FP32_KAHAN = 1 } sph_precision;

typedef struct {
    double box[3];       /* periodic box lengths (> 0); ignored by sph_batch_solve        */
    int32_t periodic;    /* 1: periodic box, minimum image (positions in [0, box));
                            0: open boundaries                                          */
    int32_t kernel;      /* sph_kernel: SPH_KERNEL_M4 (W = 8/(pi h^3) w) or
                            SPH_KERNEL_WENDLAND_C6 (W = 1365/(64 pi h^3) (1-q)^8 (1+8q+25q^2+32q^3),
                            the paper's kernel, Sec. II-B); sph_density_eval_static: M4 only */
    double nngb;         /* target weighted count (> the self term: 32/3 M4, 1365/48 C6)   */
    double tol;          /* band half-width (>= 0)                                        */
    int32_t max_iter;    /* passes, 1..64                                                  */
    int32_t precision;   /* sph_precision                                                  */
    int32_t use_graph;   /* 1: run the pass loop as a CUDA graph with a device-side loop  */
    int32_t list_entries;/* 0: none; 16..1024: keep cached neighbour lists.  Listing 1 loops
                            over a neighbour list (ngblist) built by the search; the context
                            keeps, for every particle, the particles its last search found
                            within (1 + list_margin_pct / 100) h (at most list_entries of
                            them, else no list), and a later pass of the same solve whose h
                            stays within that radius evaluates the list instead of searching
                            again.  Costs 4 * list_entries + 16 bytes of device memory per
                            particle of capacity, allocated by sph_create; fixed for the
                            context's lifetime.  The FP32 mode needs direct_pct = 0.        */
    const char *tune_cache; /* autotuner cache file, or NULL for built-in defaults         */
} sph_params;

#define SPH_MAX_PASSES 64

typedef struct {
    int32_t passes;                          /* evaluation passes run                     */
    int32_t kernel_launches;                 /* CUDA kernels of the call and of its sort  */
    int64_t todo_per_pass[SPH_MAX_PASSES];   /* particles evaluated in each pass          */
    int64_t unconverged;                     /* still off target after max_iter passes    */
    int64_t exceeded;                        /* stopped because h reached min(box)/2      */
    int64_t pair_evals;                      /* sum over passes of in-h pairs (self incl.) */
    double sort_ms;                          /* device time of the sort stage             */
    double solve_ms;                         /* device time of the solve                  */
    double density_ms;                       /* device time of the density stage of every
                                                pass: cached-list evaluation, work-item
                                                set-up and density kernels               */
    int32_t density_launches;                /* passes whose density stage was timed      */
    int32_t pad;
    int64_t pair_tests;                      /* candidate-target distance tests performed */
    int64_t pairs_per_pass[SPH_MAX_PASSES];  /* in-h pairs of each pass                   */
    double density_ms_per_pass[SPH_MAX_PASSES]; /* density-kernel time of each pass       */
    int64_t list_evals;                      /* target evaluations served by cached lists */
} sph_stats;

typedef struct sph_ctx sph_ctx;

/* Knobs of the spatial decomposition and of the density kernels' launch, set by the
 * autotuner or by hand.  They change speed, never results beyond summation order.
 * Defaults: {0, 3, 1, 0, 0, 32, 256, 0, 10, 0}. */
typedef struct {
    int32_t group_shift;  /* a work item gathers todo targets that share an octree cell of edge
                             >= h / 2^group_shift (-2..3)                                     */
    int32_t cell_div;     /* candidate cells have an edge >= (query-box extent) / cell_div, so
                             at most (cell_div + 1)^3 cells are looked up per item (1..3)     */
    int32_t table_extra;  /* dense cell-table levels beyond one cell per particle (0..1); takes
                             effect at the next sort                                          */
    int32_t direct_pct;   /* FP32 pair loop: 0 evaluates every staged candidate directly
                             (fastest measured); otherwise in-h pairs are queued per lane
                             until more than this percentage of an item's first tests fall
                             within h (1..101; 101 = always queue).  FP64 always queues.      */
    int32_t item_cap;     /* 0: a work item is a run of todo targets sharing the octree cell of
                             their grouping level; 2..64: the item is the coarsest octree cell,
                             no coarser than that level, holding at most item_cap todo targets
                             (compact items: fewer candidate tests per neighbour found)          */
    int32_t item_max;     /* targets per work item at most: 1, 2, 4, 8, 16 or 32 (a target then
                             gets at least 32 / item_max lanes of the warp)                      */
    int32_t block_threads;/* threads per block of the density kernels: 64, 128 or 256           */
    int32_t blocks_per_sm;/* resident blocks per SM of the persistent density grid, 0 = as many
                             as fit (occupancy); larger values are clamped to that              */
    int32_t list_margin_pct; /* cached neighbour lists hold the particles within
                             (1 + list_margin_pct / 100) h of the search (1..100)              */
    int32_t sparse_shift; /* group_shift used while the todo list is sparse (fewer than 1/8 of
                             the particles): the targets left late in a solve are scattered, so
                             a cell of edge up to 2h may hold targets far apart relative to their
                             h; a finer grouping keeps each item's staging ball near its
                             targets' own (-2..3)                                              */
    int32_t sparse_item_max; /* item_max used while the todo list is sparse: 0 = item_max, else 1,
                             2, 4, 8, 16 or 32.  Late in a solve the few targets left can carry h
                             so large that one item streams 10^5 candidates while the rest of
                             the GPU waits; smaller items let several warps share that work    */
} sph_tuning;

/* Create a context bound to `cuda_stream` (a cudaStream_t; NULL = legacy default stream)
 * on the current CUDA device, with scratch for up to `capacity` particles (and up to
 * `capacity` batch groups).  Allocates all device memory the context will ever use.
 * The parameters are the paper's statement of the problem (Sec. II-B with Eq. 1): the
 * kernel (Wendland C6 in the paper, M4 by default here), the target neighbour number
 * (295 in the paper) with its tolerance, the periodic box, and the recompute limit of
 * Sec. IV-A.
 * Errors: INVALID_ARG (NULL params/out, capacity < 1 or > 2^31 - 2^20, bad params),
 * CUDA (no device), OOM (device allocation failed). */
sph_status sph_create(const sph_params *params, int64_t capacity, void *cuda_stream, sph_ctx **out);

/* Replace the solve parameters of a context (precision, nngb, tol, max_iter, use_graph).
 * Changing box or periodic invalidates the sorted state (sph_sort must run again), and so
 * does switching to FP64 after a sort in FP32 (an FP32 sort keeps no FP64 records).  The
 * list_entries of a context cannot change (INVALID_ARG). */
sph_status sph_set_params(sph_ctx *ctx, const sph_params *params);

/* Read or replace the tuning of a context.  Errors: INVALID_ARG (NULL, out of range). */
sph_status sph_get_tuning(const sph_ctx *ctx, sph_tuning *out);
sph_status sph_set_tuning(sph_ctx *ctx, const sph_tuning *tuning);

/* Autotuner: the GPU counterpart of the work distribution choices of Sec. IV-A (dynamic
 * scheduling of uneven per-particle work).  Times full solves from h_dev (n doubles, caller
 * order, read only) on the particles of the last sph_sort while it varies, one knob at a
 * time from the current tuning and keeping the best value of each (two rounds): the item
 * cap (0, 16, 32, 64), targets per item (8, 16, 32), the grouping level (group_shift
 * -1..1), the candidate cell size (cell_div 2..3), threads per block (128, 256),
 * resident blocks per SM (all that fit, or one fewer), the grouping level of sparse passes
 * (sparse_shift -1..2) and, with cached lists, the list margin (5, 10, 20 %).  Keeps the fastest tuning in the
 * context and, when the context has a tune_cache file, appends it there; sph_sort applies
 * the last cached entry that matches the GPU, the particle-count bucket (floor log2 n),
 * periodic and precision.  best may be NULL.  Results never change beyond summation order.
 * Errors: as sph_density_solve. */
sph_status sph_autotune(sph_ctx *ctx, const double *h_dev, sph_tuning *best);

/* Spatially order n particles (Morton keys on 32-bit fixed-point coordinates, radix
 * sort, gather into a sorted SoA, cell tables; in FP32 the gather moves only the 16-byte
 * fixed-point records, in FP64 also the FP64 ones).  This is the spatial structure behind the
 * neighbour search: the paper's Barnes-Hut tree stored as a flat array (Sec. II-A), here an
 * octree implicit in the Morton order, and its AoS-to-SoA gather (Sec. IV-B).  The gather
 * keeps only the fields the density loop reads.  pos_xyz_dev holds three planes of n
 * doubles each (x[0..n), y[0..n), z[0..n)); mass_dev holds n doubles > 0.  Periodic
 * positions must lie in [0, box[d]) (-0.0 counts as 0); a coordinate is stored as the
 * nearest multiple of box[d] / 2^32 (ties to even; one that rounds to box[d] wraps to 0).
 * Masses must be finite and > 0.  Errors: INVALID_ARG (NULL, n < 1), OOM (n > capacity),
 * CUDA; a NaN, infinite or out-of-box position or a bad mass -> DEVICE_STATUS. */
sph_status sph_sort(sph_ctx *ctx, int64_t n, const double *pos_xyz_dev, const double *mass_dev);

/* Solve h for the particles of the last sph_sort: the recompute loop of Sec. IV-A
 * (Listing 3), each pass evaluating Eq. (1) for the particles on the todo list and
 * adjusting the h of those still outside the band.  h_inout_dev: n doubles, the starting
 * h on entry (0 < h < min(box)/2 when periodic) and the final h on exit; rho_out_dev:
 * n doubles; count_out_dev: n int32 (integer neighbour count, self included);
 * nw_out_dev: n doubles or NULL (weighted count N_w).  An unconverged particle gets the
 * last h it was evaluated at and the density/counts of that evaluation.  stats may be
 * NULL.  Returns OK, NOT_CONVERGED or H_EXCEEDS_BOX (outputs are written in all three
 * cases), or NOT_SORTED / INVALID_ARG / DEVICE_STATUS / CUDA. */
sph_status sph_density_solve(sph_ctx *ctx, double *h_inout_dev, double *rho_out_dev,
                             int32_t *count_out_dev, double *nw_out_dev, sph_stats *stats);

/* One density evaluation at fixed h (no iteration) for the particles of the last
 * sph_sort: Eq. (1) in gather form, the density loop of Listing 1 over every particle.
 * h_dev: n doubles in caller order.  Outputs (caller order): rho, integer
 * count, N_w and dN_w/dh; nw/dnw may be NULL. */
sph_status sph_density_eval(sph_ctx *ctx, const double *h_dev, double *rho_out_dev,
                            int32_t *count_out_dev, double *nw_out_dev, double *dnw_out_dev);

/* Neighbour sets of sampled particles, for checking the search itself (a test aid).
 * Listing 1 loops over a neighbour list (ngblist) of the particles within h; the GPU never
 * stores such lists, it tests staged candidates against h on the fly.  This call runs one
 * density evaluation at fixed h exactly as sph_density_eval does (the same work items,
 * staging, FP32 or FP64 distance tests and kernel instantiation apart from the recording)
 * and, for each sampled particle, records every particle j with r_ij < h_i (the particle
 * itself included), i.e. the neighbour list Eq. (1) sums over.
 *   h_dev:          n doubles, caller order (as sph_density_eval);
 *   sample_dev:     n_sample distinct caller indices in [0, n), 1 <= n_sample <= n (int64);
 *   nbr_dev:        n_sample * max_nbr int32; row k receives the caller indices of the
 *                   neighbours of sample k, in no particular order;
 *   nbr_count_dev:  n_sample int32: the number of neighbours of sample k (all of them, also
 *                   when more than max_nbr exist; only the first max_nbr are written);
 *   rho_out_dev, count_out_dev: n entries each, as sph_density_eval (count_out[sample[k]]
 *                   equals nbr_count[k]).
 * Uses context scratch only.  Errors: INVALID_ARG (NULL, n_sample outside [1, n],
 * max_nbr < 1, a sample index outside [0, n) or repeated), NOT_SORTED, UNSUPPORTED (FP32
 * with direct_pct != 0), DEVICE_STATUS (bad h), CUDA. */
sph_status sph_neighbours_sampled(sph_ctx *ctx, const double *h_dev, int64_t n_sample,
                                  const int64_t *sample_dev, int32_t max_nbr, int32_t *nbr_dev,
                                  int32_t *nbr_count_dev, double *rho_out_dev, int32_t *count_out_dev);

/* Further pair computations over the same neighbour sets: the "other particle interaction
 * computations" that Listing 1 runs inside the density loop after the density sum (the second
 * phase of the particle interactions, Sec. II-A).  The paper leaves them open; these are the
 * standard SPH velocity-field estimates, in gather form at each particle's h (typically the
 * converged h of sph_density_solve), over j with r_ij < h_i, the particle itself included:
 *   rho_i      = sum_j m_j W_ij                                  (Eq. 1)
 *   vmean_i    = (1 / rho_i) sum_j m_j W_ij v_j                  kernel-weighted mean velocity
 *   sigma2_i   = (1 / rho_i) sum_j m_j W_ij |v_j - vmean_i|^2    velocity dispersion
 *   div_i      = (1 / rho_i) sum_j m_j (v_j - v_i) . grad_i W_ij
 *   curl_i     = (1 / rho_i) sum_j m_j (v_i - v_j) x grad_i W_ij
 * with W_ij = W(r_ij, h_i) and grad_i W_ij = dW/dr(r_ij) (r_i - r_j) / r_ij (zero at r = 0).
 *   h_dev:             n doubles, caller order, each in (0, min(box)/2) when periodic;
 *   vel_xyz_dev:       3 x n doubles, caller order (x block, y block, z block);
 *   rho_out_dev, sigma2_out_dev, div_out_dev: n doubles; vmean_xyz_out_dev, curl_xyz_out_dev:
 *                      3 x n doubles (x, y, z blocks); count_out_dev: n int32 (#{r_ij < h_i});
 *   stats (nullable):  passes = 1, pair_evals (in-h pairs), pair_tests, solve_ms (the call) and
 *                      density_ms (work-item set-up and the interaction kernel).
 * FP64 precision: the neighbour test and every pair term in FP64 from the FP64 positions and
 * velocities.  FP32_KAHAN: FP32 offsets, velocities and pair terms with compensated sums.
 * Uses context memory only (32 bytes of velocity records per particle of capacity).
 * Errors: INVALID_ARG (NULL), NOT_SORTED, DEVICE_STATUS (bad h, non-finite velocity), CUDA. */
sph_status sph_interact(sph_ctx *ctx, const double *h_dev, const double *vel_xyz_dev, double *rho_out_dev,
                        double *vmean_xyz_out_dev, double *sigma2_out_dev, double *div_out_dev,
                        double *curl_xyz_out_dev, int32_t *count_out_dev, sph_stats *stats);

/* k-nearest-neighbour smoothing lengths: the Subfind form of the density loop (Sec. IV-D and
 * Listing 3), where each particle's neighbour list is put in order of distance and its K
 * nearest entries interact.  For every particle of the last sph_sort:
 *   h_i     = distance to the K-th nearest particle, the particle itself counted first;
 *   rho_i   = Eq. (1) at h_i (the K-th neighbour sits at q = 1 and adds nothing, so equal
 *             distances do not change it);
 *   count_i = #{j : r_ij^2 < h_i^2}: K - 1, or more when other particles sit at distance h_i
 *             or h_i^2 rounds above the K-th squared distance;  nw_i = N_w(h_i) (nullable).
 * h_inout_dev (n doubles, caller order): a starting search radius on entry (below min(box)/2;
 * it steers the passes, not the result), or <= 0 to have one estimated from the local cell
 * density; h_i on exit.  Each pass streams a target's candidates inside its radius through
 * a per-warp buffer of 896 squared distances that is cut back to its
 * K nearest whenever it would overflow; with at least K inside the radius the K-th is
 * selected (radix select), otherwise the radius grows (count ~ radius^3) and the target
 * returns in the next pass, for at most max_iter passes.
 * FP64 forms every distance exactly as the FP64 density pairs; FP32 from the FP32 offsets.
 * Needs 2 <= k <= SPH_KNN_MAX_K and k <= n.  Returns OK; NOT_CONVERGED (passes ran out);
 * H_EXCEEDS_BOX (the K-th distance, or the radius that would hold K particles, reaches
 * min(box)/2); those particles report their last radius and the density there.  Errors:
 * INVALID_ARG, NOT_SORTED (no sph_sort since the context was created or since the last
 * sph_batch_solve, which leaves groups, not one sorted set), DEVICE_STATUS, CUDA.
 * stats: passes/todo_per_pass/density_ms of the selection passes, pair_tests = candidates
 * streamed, pair_evals / pairs_per_pass = neighbour-list entries (squared distances inside
 * the search radius) built by the selection passes, unconverged, exceeded. */
#define SPH_KNN_MAX_K 512
sph_status sph_knn_solve(sph_ctx *ctx, int32_t k, double *h_inout_dev, double *rho_out_dev,
                         int32_t *count_out_dev, double *nw_out_dev, sph_stats *stats);

/* Solve many independent non-periodic groups in one pass loop: the recompute loop of
 * Sec. IV-A (Listing 3) with Eq. (1), run over many independent particle sets at once, each
 * with its own neighbour target and tolerance (Sec. II-B).  Group g owns the
 * particles [offsets[g], offsets[g+1]) of the flattened arrays; offsets_dev holds
 * n_groups + 1 int64 (offsets[0] = 0, non-decreasing); nngb_dev and tol_dev hold one
 * double per group.  pos_xyz_dev is three planes of n = offsets[n_groups] doubles.
 * Every group is sorted, searched and iterated on its own (no box, no h limit), but all
 * groups share each kernel launch.  Returns like sph_density_solve. */
sph_status sph_batch_solve(sph_ctx *ctx, int64_t n_groups, const int64_t *offsets_dev,
                           const double *pos_xyz_dev, const double *mass_dev,
                           const double *nngb_dev, const double *tol_dev, double *h_inout_dev,
                           double *rho_out_dev, int32_t *count_out_dev, double *nw_out_dev,
                           sph_stats *stats);

/* ---- Evaluation without any device allocation -------------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that must not call
 * cudaMalloc/cudaFree themselves or through this library: a plugin inside a host program
 * that owns all device memory through its own pool, or a latency-critical loop where
 * cudaFree would stall every stream on the device.
 *
 * It performs sph_sort followed by sph_density_eval (fixed h, one density pass) for up to
 * SPH_STATIC_MAX_PARTICLES periodic particles, with every intermediate buffer placed in one
 * fixed array of device memory compiled into the library (about 5 MB, reserved on every GPU
 * that loads the library until the process exits).  No context is involved; params gives
 * box, periodic (must be 1), kernel (M4), precision; nngb/tol/max_iter/use_graph are unused.
 * pos_xyz_dev (three planes of n doubles), mass_dev and h_dev are inputs in caller order;
 * rho/count (required) and nw/dnw (nullable) are outputs in caller order; all are device
 * memory owned by the caller.  Work runs on cuda_stream and the call returns after the
 * stream has finished it.
 * The first call on each device looks up the array's device address; make that first call
 * before any stream capture.  Every call reuses the same array, so calls whose GPU work
 * overlaps (other streams, other host threads) race and must be serialised by the caller.
 * Errors: INVALID_ARG (NULL pointers, n < 1, bad box or precision), OOM (n greater than
 * SPH_STATIC_MAX_PARTICLES; nothing is allocated instead), UNSUPPORTED (open boundaries or
 * another kernel), CUDA, DEVICE_STATUS (bad positions, masses or h). */
#define SPH_STATIC_MAX_PARTICLES 32768
sph_status sph_density_eval_static(const sph_params *params, int64_t n, const double *pos_xyz_dev,
                                   const double *mass_dev, const double *h_dev, void *cuda_stream,
                                   double *rho_out_dev, int32_t *count_out_dev,
                                   double *nw_out_dev, double *dnw_out_dev);

/* Release every resource of the context (NULL is ignored). */
void sph_destroy(sph_ctx *ctx);

/* Static description of a status code. */
const char *sph_status_string(sph_status status);

/* One-line description of the last error on the context ("" if none). */
const char *sph_last_error(const sph_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
