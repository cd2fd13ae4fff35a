/*
 * sph_oracle.c -- plain FP64 CPU oracle for the SPH density / smoothing-length solve.
 *
 * TEST INFRASTRUCTURE ONLY.  The CUDA library never links, loads or calls this file.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (Baruffa et al., "Performance Optimisation of SPH Algorithms for
 * Multi/Many-Core Architectures", arXiv:1612.06090):
 *
 *  - Density by kernel interpolation, Eq. (1): rho_i = sum_j m_j W(|r_i - r_j|, h).
 *    Read in gather form: the smoothing length of the target particle i is used for
 *    every pair (the printed equation carries h_j; see the readings list).
 *    The self pair j = i is included.  A neighbour is a particle with r_ij < h, strictly.
 *  - Kernel W: M4 cubic spline in 3-D with compact support h (or the paper's Wendland C6,
 *    selected by the `kernel` argument; see oracle_w_c6),
 *    W(r, h) = 8 / (pi h^3) w(q), q = r / h,
 *    w = 1 - 6 q^2 + 6 q^3 (q <= 1/2), 2 (1 - q)^3 (1/2 < q < 1), 0 otherwise.
 *    (The paper runs a Wendland C6 kernel with 295 neighbours, Sec. II-B; this solve
 *    uses the M4 kernel with a target of Nngb weighted neighbours.)
 *  - Weighted neighbour count N_w(h) = (4 pi / 3) h^3 sum_j W(r_ij, h) = (32/3) sum_j w(q_j)
 *    and its derivative dN_w/dh = (32/3)(1/h) sum_j (-q_j w'(q_j)).
 *  - The iteration of Sec. IV-A (Listings 2 and 3): particles whose neighbour count is
 *    off target get a new h and are recomputed; each pass runs only over the "todo"
 *    list of still-unconverged particles, spread over OpenMP threads with dynamic
 *    scheduling (the "lockless" scheme).  The paper gives no h-update rule; this one is:
 *      converged      iff |N_w - Nngb| <= tol (outputs come from that same evaluation);
 *      bracket        N_w < Nngb -> h_lo = h, else h_hi = h;
 *      Newton         h' = h - (N_w - Nngb) / N_w', accepted iff N_w' > 0,
 *                     h_lo < h' < h_hi and h/2 <= h' <= 2h;
 *      fallback       both bounds set -> (h_lo + h_hi) / 2; only h_lo -> h * 2^(1/3);
 *                     only h_hi -> h / 2^(1/3) (the double literal 1.2599210498948732);
 *      box limit      periodic and h' >= min(box) / 2 -> the particle stops with
 *                     status "h exceeds box";
 *      pass limit     after max_iter evaluations -> status "not converged".
 *    An unconverged particle reports the last h it was evaluated at, with the density
 *    and counts of that evaluation.
 *  - The k-nearest-neighbour form of h (Sec. IV-D): h_i = distance to the K-th nearest
 *    particle, rho_i by Eq. (1) at that h (oracle_knn).
 *  - Further pair computations over the same neighbour sets (the "other particle
 *    interactions" of Listing 1): kernel-weighted mean velocity, velocity dispersion,
 *    velocity divergence and curl at the converged h (oracle_interact).
 *
 * Neighbour search: a stack of uniform FP64 bucket grids (cell size box / 2^k).  For a
 * target with smoothing length h the grid with the coarsest cells no larger than h is
 * used and every bucket meeting [x - h, x + h] is scanned.  Buckets are row-major cell
 * ids sorted with qsort and looked up with binary search.  A brute-force O(N) scan per
 * target is also provided; the two are cross-checked by the tests.
 *
 * Build with -ffp-contract=off so that every product and sum rounds separately.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_LEVEL 20 /* 2^60 cell ids still fit an int64 */
#define ORACLE_MAX_PASSES 64
#define ORACLE_GROWTH 1.2599210498948732 /* 2^(1/3) as the double literal of the readings */

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_EXCEEDS_BOX = 2 };

/* ------------------------------------------------------------------------------------ */
/* Kernel                                                                                */
/* ------------------------------------------------------------------------------------ */

/* Dimensionless M4 shape w(q); W = 8/(pi h^3) w(q). */
double oracle_w(double q)
{
    if (q <= 0.5) {
        double t = 6.0 * q - 6.0;
        return 1.0 + (q * q) * t;
    }
    if (q < 1.0) {
        double a = 1.0 - q;
        return 2.0 * (a * a * a);
    }
    return 0.0;
}

/* Wendland C6 shape (the kernel of Sec. II-B, 295 neighbours) with compact support h:
 * W(r, h) = 1365 / (64 pi h^3) w(q), w = (1 - q)^8 (1 + 8 q + 25 q^2 + 32 q^3) for q < 1. */
double oracle_w_c6(double q)
{
    if (q < 1.0) {
        double a = 1.0 - q;
        double a2 = a * a;
        double a4 = a2 * a2;
        double a8 = a4 * a4;
        double p = 1.0 + q * (8.0 + q * (25.0 + q * 32.0));
        return a8 * p;
    }
    return 0.0;
}

/* -q w'(q) of the Wendland C6 shape: 22 q^2 (1 - q)^7 (1 + 7 q + 16 q^2). */
double oracle_mqdw_c6(double q)
{
    if (q < 1.0) {
        double a = 1.0 - q;
        double a2 = a * a;
        double a4 = a2 * a2;
        double a7 = a4 * a2 * a;
        double p = 1.0 + q * (7.0 + q * 16.0);
        return 22.0 * (q * q) * a7 * p;
    }
    return 0.0;
}

/* -q w'(q), the term whose sum gives dN_w/dh. */
double oracle_mqdw(double q)
{
    if (q <= 0.5) {
        return (q * q) * (12.0 - 18.0 * q);
    }
    if (q < 1.0) {
        double a = 1.0 - q;
        return (6.0 * q) * (a * a);
    }
    return 0.0;
}

/* ------------------------------------------------------------------------------------ */
/* Particle set and bucket grids                                                         */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    const double *x, *y, *z, *m;
    int periodic;
    double box[3];    /* periodic box lengths */
    double origin[3]; /* non-periodic: bounding-box minimum */
    double ext[3];    /* periodic: box; non-periodic: one cubic extent for all three */
    int kernel;       /* 0: M4 cubic spline, 1: Wendland C6 */
} pset;

typedef struct {
    int built;
    int64_t g;        /* cells per dimension, 2^level */
    double cell[3];   /* cell size per dimension */
    int64_t *ids;     /* sorted cell ids */
    int64_t *order;   /* particle index for each sorted entry */
} bucket_grid;

typedef struct {
    int64_t id, idx;
} id_idx;

static int cmp_id_idx(const void *a, const void *b)
{
    const id_idx *p = (const id_idx *)a, *q = (const id_idx *)b;
    if (p->id < q->id) return -1;
    if (p->id > q->id) return 1;
    if (p->idx < q->idx) return -1;
    if (p->idx > q->idx) return 1;
    return 0;
}

static int64_t cell_coord(double x, double origin, double cell, int64_t g)
{
    double f = floor((x - origin) / cell);
    if (f < 0.0) return 0;
    if (f > (double)(g - 1)) return g - 1;
    return (int64_t)f;
}

static int build_grid(const pset *ps, int level, bucket_grid *bg)
{
    int64_t n = ps->n, g = (int64_t)1 << level;
    bg->g = g;
    for (int d = 0; d < 3; d++) bg->cell[d] = ps->ext[d] / (double)g;
    id_idx *tmp = (id_idx *)malloc((size_t)(n > 0 ? n : 1) * sizeof(id_idx));
    bg->ids = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    bg->order = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!tmp || !bg->ids || !bg->order) {
        free(tmp);
        free(bg->ids);
        free(bg->order);
        bg->ids = bg->order = NULL;
        return -1;
    }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t ix = cell_coord(ps->x[i], ps->origin[0], bg->cell[0], g);
        int64_t iy = cell_coord(ps->y[i], ps->origin[1], bg->cell[1], g);
        int64_t iz = cell_coord(ps->z[i], ps->origin[2], bg->cell[2], g);
        tmp[i].id = ix + g * (iy + g * iz);
        tmp[i].idx = i;
    }
    qsort(tmp, (size_t)n, sizeof(id_idx), cmp_id_idx);
    for (int64_t i = 0; i < n; i++) {
        bg->ids[i] = tmp[i].id;
        bg->order[i] = tmp[i].idx;
    }
    free(tmp);
    bg->built = 1;
    return 0;
}

static void free_grid(bucket_grid *bg)
{
    free(bg->ids);
    free(bg->order);
    memset(bg, 0, sizeof(*bg));
}

/* First sorted position whose id is >= key. */
static int64_t lower_bound_id(const int64_t *ids, int64_t n, int64_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ids[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

/* Coarsest grid level whose cells are no larger than h in every dimension. */
static int level_for(const pset *ps, double h)
{
    double emax = ps->ext[0];
    if (ps->ext[1] > emax) emax = ps->ext[1];
    if (ps->ext[2] > emax) emax = ps->ext[2];
    int k = 0;
    while (k < ORACLE_MAX_LEVEL && emax / (double)((int64_t)1 << k) > h) k++;
    return k;
}

/* ------------------------------------------------------------------------------------ */
/* One density evaluation at fixed h                                                     */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double sum_mw, sum_w, sum_dw; /* sum m_j w_j, sum w_j, sum -q_j w'(q_j) */
    int64_t count;                /* #{j : r_ij < h} */
    int64_t near;                 /* #{j : |r_ij - h| <= near_rel * h} */
} acc_t;

static inline double min_image(double dx, double L)
{
    if (dx > 0.5 * L) return dx - L;
    if (dx < -0.5 * L) return dx + L;
    return dx;
}

static inline void pair(const pset *ps, int64_t i, int64_t j, double h, double h2,
                        double near_rel, acc_t *a)
{
    double dx = ps->x[j] - ps->x[i];
    double dy = ps->y[j] - ps->y[i];
    double dz = ps->z[j] - ps->z[i];
    if (ps->periodic) {
        dx = min_image(dx, ps->box[0]);
        dy = min_image(dy, ps->box[1]);
        dz = min_image(dz, ps->box[2]);
    }
    double r2 = dx * dx + dy * dy + dz * dz;
    if (near_rel > 0.0) {
        double r = sqrt(r2);
        if (fabs(r - h) <= near_rel * h) a->near++;
    }
    if (r2 < h2) {
        double r = sqrt(r2);
        double q = r / h;
        double w = ps->kernel ? oracle_w_c6(q) : oracle_w(q);
        a->sum_mw += ps->m[j] * w;
        a->sum_w += w;
        a->sum_dw += ps->kernel ? oracle_mqdw_c6(q) : oracle_mqdw(q);
        a->count++;
    }
}

static void eval_brute(const pset *ps, int64_t i, double h, double near_rel, acc_t *a)
{
    double h2 = h * h;
    memset(a, 0, sizeof(*a));
    for (int64_t j = 0; j < ps->n; j++) pair(ps, i, j, h, h2, near_rel, a);
}

/* First bucket and bucket count per dimension of the buckets meeting [x_i - h, x_i + h]
 * (a periodic row that the interval covers entirely is taken once, from bucket 0). */
static void bucket_box(const pset *ps, const bucket_grid *bg, const double xi[3], double h,
                       int64_t lo[3], int64_t cnt[3])
{
    int64_t g = bg->g;
    for (int d = 0; d < 3; d++) {
        double c = bg->cell[d];
        int64_t a0 = (int64_t)floor((xi[d] - h - ps->origin[d]) / c);
        int64_t a1 = (int64_t)floor((xi[d] + h - ps->origin[d]) / c);
        if (ps->periodic) {
            if (a1 - a0 + 1 >= g) { /* the whole periodic row, each bucket once */
                lo[d] = 0;
                cnt[d] = g;
            } else {
                lo[d] = a0;
                cnt[d] = a1 - a0 + 1;
            }
        } else {
            if (a0 < 0) a0 = 0;
            if (a1 > g - 1) a1 = g - 1;
            lo[d] = a0;
            cnt[d] = a1 >= a0 ? a1 - a0 + 1 : 0;
        }
    }
}

/* Scan every bucket meeting [x_i - h, x_i + h] in each dimension. */
static void eval_grid(const pset *ps, const bucket_grid *bg, int64_t i, double h,
                      double near_rel, acc_t *a)
{
    double h2 = h * h;
    const double xi[3] = {ps->x[i], ps->y[i], ps->z[i]};
    int64_t lo[3], cnt[3];
    int64_t g = bg->g;
    memset(a, 0, sizeof(*a));
    bucket_box(ps, bg, xi, h, lo, cnt);
    for (int64_t kz = 0; kz < cnt[2]; kz++) {
        int64_t cz = lo[2] + kz;
        if (ps->periodic) cz = ((cz % g) + g) % g;
        for (int64_t ky = 0; ky < cnt[1]; ky++) {
            int64_t cy = lo[1] + ky;
            if (ps->periodic) cy = ((cy % g) + g) % g;
            for (int64_t kx = 0; kx < cnt[0]; kx++) {
                int64_t cx = lo[0] + kx;
                if (ps->periodic) cx = ((cx % g) + g) % g;
                int64_t id = cx + g * (cy + g * cz);
                int64_t s = lower_bound_id(bg->ids, ps->n, id);
                for (int64_t p = s; p < ps->n && bg->ids[p] == id; p++)
                    pair(ps, i, bg->order[p], h, h2, near_rel, a);
            }
        }
    }
}

/* rho = sigma h^-3 sum m w; N_w = (4 pi / 3) sigma sum w; dN_w/dh = (4 pi / 3) sigma h^-1 sum -q w'
 * with sigma = 8/pi (M4) or 1365/(64 pi) (Wendland C6), i.e. (4 pi / 3) sigma = 32/3 or 1365/48. */
static void finish(int kernel, double h, const acc_t *a, double *rho, double *nw, double *dnw)
{
    const double pi = 3.14159265358979323846;
    if (kernel) {
        *rho = a->sum_mw * (1365.0 / (64.0 * pi * h * h * h));
        *nw = (1365.0 / 48.0) * a->sum_w;
        *dnw = (1365.0 / 48.0) * a->sum_dw / h;
    } else {
        *rho = a->sum_mw * (8.0 / (pi * h * h * h));
        *nw = (32.0 / 3.0) * a->sum_w;
        *dnw = (32.0 / 3.0) * a->sum_dw / h;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Particle-set setup                                                                    */
/* ------------------------------------------------------------------------------------ */

static void setup_pset(pset *ps, int64_t n, const double *x, const double *y, const double *z,
                       const double *m, const double *box, int periodic, int kernel)
{
    memset(ps, 0, sizeof(*ps));
    ps->kernel = kernel;
    ps->n = n;
    ps->x = x;
    ps->y = y;
    ps->z = z;
    ps->m = m;
    ps->periodic = periodic;
    if (periodic) {
        for (int d = 0; d < 3; d++) {
            ps->box[d] = box[d];
            ps->origin[d] = 0.0;
            ps->ext[d] = box[d];
        }
    } else {
        double lo[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL}, hi[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL};
        const double *c[3] = {x, y, z};
        for (int64_t i = 0; i < n; i++)
            for (int d = 0; d < 3; d++) {
                if (c[d][i] < lo[d]) lo[d] = c[d][i];
                if (c[d][i] > hi[d]) hi[d] = c[d][i];
            }
        double e = 0.0;
        for (int d = 0; d < 3; d++)
            if (n > 0 && hi[d] - lo[d] > e) e = hi[d] - lo[d];
        if (e <= 0.0) e = 1.0;
        e *= 1.0000001; /* keep the maximum inside the last bucket */
        for (int d = 0; d < 3; d++) {
            ps->origin[d] = n > 0 ? lo[d] : 0.0;
            ps->ext[d] = e;
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Public entry points                                                                   */
/* ------------------------------------------------------------------------------------ */

/* Fixed-h evaluation for the targets listed in `targets` (NULL: all particles).
 * Outputs are indexed by target position.  mode 0 = bucket grids, 1 = brute force.
 * near_rel > 0 also counts pairs with |r - h| <= near_rel * h into near_out. */
int oracle_eval(int64_t n, const double *x, const double *y, const double *z, const double *m,
                const double *box, int periodic, int64_t n_targets, const int64_t *targets,
                const double *h, int mode, double near_rel, double *rho, double *nw, double *dnw,
                int64_t *count, int64_t *near_out, int kernel)
{
    pset ps;
    setup_pset(&ps, n, x, y, z, m, box, periodic, kernel);
    if (n_targets < 0) n_targets = n;
    bucket_grid grids[ORACLE_MAX_LEVEL + 1];
    memset(grids, 0, sizeof(grids));
    if (mode == 0) {
        for (int64_t t = 0; t < n_targets; t++) {
            int k = level_for(&ps, h[t]);
            if (!grids[k].built && build_grid(&ps, k, &grids[k]) != 0) return -1;
        }
    }
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_targets; t++) {
        int64_t i = targets ? targets[t] : t;
        acc_t a;
        if (mode == 0) eval_grid(&ps, &grids[level_for(&ps, h[t])], i, h[t], near_rel, &a);
        else eval_brute(&ps, i, h[t], near_rel, &a);
        finish(ps.kernel, h[t], &a, &rho[t], &nw[t], &dnw[t]);
        count[t] = a.count;
        if (near_out) near_out[t] = a.near;
    }
    for (int k = 0; k <= ORACLE_MAX_LEVEL; k++)
        if (grids[k].built) free_grid(&grids[k]);
    return 0;
}

/* One step of the h iteration for a particle evaluated at h = hc that is not yet in the
 * band: the bracket takes hc (below the target -> lower bound, else upper bound; an unset
 * lower bound is 0, an unset upper bound +inf), then the Newton point
 * hc - (N_w - Nngb) / N_w' is returned when N_w' > 0 and it lies strictly inside the
 * bracket and within [hc/2, 2 hc]; otherwise the bracket midpoint when both bounds are
 * set, hc * 2^(1/3) with only a lower bound, hc / 2^(1/3) with only an upper bound. */
double oracle_h_update(double hc, double nw, double dnw, double nngb, double *hlo, double *hhi)
{
    if (nw < nngb) *hlo = hc;
    else *hhi = hc;
    if (dnw > 0.0) {
        double hn = hc - (nw - nngb) / dnw;
        if (hn > *hlo && hn < *hhi && hn >= 0.5 * hc && hn <= 2.0 * hc) return hn;
    }
    int has_lo = *hlo > 0.0, has_hi = *hhi < HUGE_VAL;
    if (has_lo && has_hi) return 0.5 * (*hlo + *hhi);
    if (has_lo) return hc * ORACLE_GROWTH;
    return hc / ORACLE_GROWTH;
}

/* Solve statistics, mirrored by a ctypes structure in oracle/__init__.py. */
typedef struct {
    int32_t passes;
    int32_t pad;
    int64_t todo_per_pass[ORACLE_MAX_PASSES];
    int64_t unconverged;
    int64_t exceeded;
    int64_t pair_evals;
} oracle_stats;

/* One smoothing-length solve over one particle set for the listed targets.
 * h_inout holds the starting h per target on entry and the last evaluated h on exit.
 * status_out per target: 0 converged, 1 not converged, 2 h exceeds box. */
static int solve_set(const pset *ps, int64_t n_targets, const int64_t *targets, double nngb,
                     double tol, int max_iter, int mode, double *h_inout, double *rho_out,
                     double *nw_out, int64_t *count_out, int32_t *status_out,
                     oracle_stats *st)
{
    size_t cap = (size_t)(n_targets > 0 ? n_targets : 1);
    double *h = (double *)malloc(cap * sizeof(double));     /* h for the next evaluation */
    double *hlo = (double *)malloc(cap * sizeof(double));
    double *hhi = (double *)malloc(cap * sizeof(double));
    int64_t *todo = (int64_t *)malloc(cap * sizeof(int64_t));
    int32_t *again = (int32_t *)malloc(cap * sizeof(int32_t));
    if (!h || !hlo || !hhi || !todo || !again) {
        free(h); free(hlo); free(hhi); free(todo); free(again);
        return -1;
    }
    bucket_grid grids[ORACLE_MAX_LEVEL + 1];
    memset(grids, 0, sizeof(grids));
    double half_box = 0.5 * fmin(ps->box[0], fmin(ps->box[1], ps->box[2]));

    int64_t ntodo = n_targets;
    for (int64_t t = 0; t < n_targets; t++) {
        h[t] = h_inout[t];
        hlo[t] = 0.0;
        hhi[t] = HUGE_VAL;
        todo[t] = t;
        again[t] = 0;
        status_out[t] = ORC_NOT_CONVERGED;
    }
    int pass = 0;
    int rc = 0;
    while (ntodo > 0 && pass < max_iter) {
        if (pass < ORACLE_MAX_PASSES) st->todo_per_pass[pass] = ntodo;
        if (mode == 0) {
            for (int64_t k = 0; k < ntodo && rc == 0; k++) {
                int lv = level_for(ps, h[todo[k]]);
                if (!grids[lv].built && build_grid(ps, lv, &grids[lv]) != 0) rc = -1;
            }
            if (rc) break;
        }
        int64_t pairs = 0;
        /* The lockless scheme: dynamic scheduling over the todo list only. */
        #pragma omp parallel for schedule(dynamic, 16) reduction(+ : pairs)
        for (int64_t k = 0; k < ntodo; k++) {
            int64_t t = todo[k];
            int64_t i = targets ? targets[t] : t;
            double hc = h[t];
            acc_t a;
            if (mode == 0) eval_grid(ps, &grids[level_for(ps, hc)], i, hc, 0.0, &a);
            else eval_brute(ps, i, hc, 0.0, &a);
            double rho, nw, dnw;
            finish(ps->kernel, hc, &a, &rho, &nw, &dnw);
            pairs += a.count;
            h_inout[t] = hc; /* outputs always describe the last evaluation */
            rho_out[t] = rho;
            nw_out[t] = nw;
            count_out[t] = a.count;
            again[t] = 0;
            if (fabs(nw - nngb) <= tol) {
                status_out[t] = ORC_OK;
                continue;
            }
            double hn = oracle_h_update(hc, nw, dnw, nngb, &hlo[t], &hhi[t]);
            if (ps->periodic && hn >= half_box) {
                status_out[t] = ORC_EXCEEDS_BOX;
                continue;
            }
            h[t] = hn;
            again[t] = 1;
        }
        if (rc) break;
        st->pair_evals += pairs;
        /* mark_for_recomputation: the next todo list keeps the unconverged, in order */
        int64_t nn = 0;
        for (int64_t k = 0; k < ntodo; k++)
            if (again[todo[k]]) todo[nn++] = todo[k];
        ntodo = nn;
        pass++;
    }
    st->passes = pass;
    int64_t unconv = 0, exc = 0;
    for (int64_t t = 0; t < n_targets; t++) {
        if (status_out[t] == ORC_NOT_CONVERGED) unconv++;
        if (status_out[t] == ORC_EXCEEDS_BOX) exc++;
    }
    st->unconverged += unconv;
    st->exceeded += exc;
    for (int k = 0; k <= ORACLE_MAX_LEVEL; k++)
        if (grids[k].built) free_grid(&grids[k]);
    free(h); free(hlo); free(hhi); free(todo); free(again);
    return rc;
}

/* Periodic (or single non-periodic) solve for the listed targets (NULL: all). */
int oracle_solve(int64_t n, const double *x, const double *y, const double *z, const double *m,
                 const double *box, int periodic, double nngb, double tol, int max_iter,
                 int64_t n_targets, const int64_t *targets, int mode, double *h_inout,
                 double *rho, double *nw, int64_t *count, int32_t *status, oracle_stats *st,
                 int kernel)
{
    pset ps;
    setup_pset(&ps, n, x, y, z, m, box, periodic, kernel);
    if (n_targets < 0) n_targets = n;
    memset(st, 0, sizeof(*st));
    return solve_set(&ps, n_targets, targets, nngb, tol, max_iter, mode, h_inout, rho, nw, count,
                     status, st);
}

/* Batch of independent non-periodic groups; group g owns [offsets[g], offsets[g+1]).
 * All arrays are flattened in group order; per-group nngb and tol. */
int oracle_batch_solve(int64_t n_groups, const int64_t *offsets, const double *x, const double *y,
                       const double *z, const double *m, const double *nngb, const double *tol,
                       int max_iter, int mode, double *h_inout, double *rho, double *nw,
                       int64_t *count, int32_t *status, oracle_stats *st, int kernel)
{
    memset(st, 0, sizeof(*st));
    const double nobox[3] = {0.0, 0.0, 0.0};
    for (int64_t g = 0; g < n_groups; g++) {
        int64_t s = offsets[g], e = offsets[g + 1];
        if (e <= s) continue;
        pset ps;
        setup_pset(&ps, e - s, x + s, y + s, z + s, m + s, nobox, 0, kernel);
        oracle_stats gs;
        memset(&gs, 0, sizeof(gs));
        int rc = solve_set(&ps, e - s, NULL, nngb[g], tol[g], max_iter, mode, h_inout + s, rho + s,
                           nw + s, count + s, status + s, &gs);
        if (rc) return rc;
        if (gs.passes > st->passes) st->passes = gs.passes;
        for (int p = 0; p < ORACLE_MAX_PASSES; p++) st->todo_per_pass[p] += gs.todo_per_pass[p];
        st->unconverged += gs.unconverged;
        st->exceeded += gs.exceeded;
        st->pair_evals += gs.pair_evals;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* k-nearest-neighbour smoothing length (Sec. IV-D)                                       */
/* ------------------------------------------------------------------------------------ */

static int cmp_double(const void *a, const void *b)
{
    const double p = *(const double *)a, q = *(const double *)b;
    return p < q ? -1 : p > q ? 1 : 0;
}

/* The Subfind form of the density loop (Listing 1 inside the loop of Listing 3, with the
 * selection of Sec. IV-D): the neighbour list of a particle is put in order of distance
 * and its first K entries are the ones that interact.  Read as a definition:
 *   h_i   = the K-th smallest of the distances r_ij over all j, the particle itself
 *           included (r_ii = 0 is the first), with r_ij the minimum-image distance when
 *           periodic and r_ij^2 formed exactly as in pair();
 *   rho_i = Eq. (1) at h = h_i; every particle with r_ij < h_i is among the K nearest and
 *           the K-th lies at q = 1, where W = 0, so equal distances do not matter;
 *   count_i = #{j : r_ij^2 < h_i^2}: K - 1, or more when other particles sit at distance h_i
 *           or when h_i^2 rounds above the K-th squared distance.
 * Every squared distance of the target is computed and the list is sorted (qsort); a
 * periodic h_i >= min(box)/2 gets status 2 (EXCEEDS_BOX) and no density.
 * K must lie in [2, n].  mode 0 evaluates the density with the bucket grids, mode 1 by
 * brute force.  status_out: 0 done, 2 exceeds box. */
int oracle_knn(int64_t n, const double *x, const double *y, const double *z, const double *m,
               const double *box, int periodic, int k, int64_t n_targets, const int64_t *targets,
               int mode, double *h_out, double *rho_out, double *nw_out, int64_t *count_out,
               int32_t *status_out, int kernel)
{
    if (k < 2 || (int64_t)k > n) return -2;
    pset ps;
    setup_pset(&ps, n, x, y, z, m, box, periodic, kernel);
    if (n_targets < 0) n_targets = n;
    int failed = 0;
    #pragma omp parallel
    {
        double *r2 = (double *)malloc((size_t)n * sizeof(double));
        if (!r2) {
            #pragma omp atomic write
            failed = 1;
        }
        #pragma omp for schedule(dynamic, 4)
        for (int64_t t = 0; t < n_targets; t++) {
            if (!r2) continue;
            const int64_t i = targets ? targets[t] : t;
            for (int64_t j = 0; j < n; j++) {
                double dx = ps.x[j] - ps.x[i];
                double dy = ps.y[j] - ps.y[i];
                double dz = ps.z[j] - ps.z[i];
                if (ps.periodic) {
                    dx = min_image(dx, ps.box[0]);
                    dy = min_image(dy, ps.box[1]);
                    dz = min_image(dz, ps.box[2]);
                }
                r2[j] = dx * dx + dy * dy + dz * dz;
            }
            qsort(r2, (size_t)n, sizeof(double), cmp_double);
            h_out[t] = sqrt(r2[k - 1]);
            status_out[t] = 0;
            if (ps.periodic) {
                double half = 0.5 * fmin(ps.box[0], fmin(ps.box[1], ps.box[2]));
                if (h_out[t] >= half) status_out[t] = ORC_EXCEEDS_BOX;
            }
        }
        free(r2);
    }
    if (failed) return -1;
    /* density at the selected h (targets whose h exceeds the box are skipped) */
    bucket_grid grids[ORACLE_MAX_LEVEL + 1];
    memset(grids, 0, sizeof(grids));
    if (mode == 0) {
        for (int64_t t = 0; t < n_targets; t++) {
            if (status_out[t] != 0) continue;
            int lv = level_for(&ps, h_out[t]);
            if (!grids[lv].built && build_grid(&ps, lv, &grids[lv]) != 0) return -1;
        }
    }
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_targets; t++) {
        if (status_out[t] != 0) {
            rho_out[t] = nw_out[t] = 0.0;
            count_out[t] = 0;
            continue;
        }
        const int64_t i = targets ? targets[t] : t;
        acc_t a;
        double dnw;
        if (mode == 0) eval_grid(&ps, &grids[level_for(&ps, h_out[t])], i, h_out[t], 0.0, &a);
        else eval_brute(&ps, i, h_out[t], 0.0, &a);
        finish(ps.kernel, h_out[t], &a, &rho_out[t], &nw_out[t], &dnw);
        count_out[t] = a.count;
    }
    for (int lv = 0; lv <= ORACLE_MAX_LEVEL; lv++)
        if (grids[lv].built) free_grid(&grids[lv]);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Other particle interactions (the second phase of Listing 1)                           */
/* ------------------------------------------------------------------------------------ */

/* The paper's density loop leaves a place for further pair computations over the same
 * neighbours ("other particle interaction computations"; Sec. II-A calls this the second
 * phase of the particle interactions) without fixing them.  The ones taken here are the
 * standard SPH velocity-field estimates over the neighbour set of Eq. (1), gather form,
 * at the target's converged h:
 *   rho_i         = sum_j m_j W_ij                                   (Eq. 1)
 *   vbar_i        = (1 / rho_i) sum_j m_j W_ij v_j                   kernel-weighted mean
 *   sigma2_i      = (1 / rho_i) sum_j m_j W_ij |v_j - vbar_i|^2      velocity dispersion
 *   (div v)_i     = (1 / rho_i) sum_j m_j (v_j - v_i) . grad_i W_ij
 *   (curl v)_i    = (1 / rho_i) sum_j m_j (v_i - v_j) x grad_i W_ij
 * with W_ij = W(r_ij, h_i) and grad_i W_ij = dW/dr (r_ij) (r_i - r_j) / r_ij, zero at
 * r_ij = 0 (the kernel is flat there); dW/dr = sigma h^-4 w'(q) and w'(q) = -mqdw(q) / q.
 * The neighbours are j with r_ij < h_i, the self pair included, r_i - r_j the minimum image
 * when periodic, all formed as in pair().  The mean is taken first and the dispersion
 * about it in a second sweep over the list, as the definition reads.
 * Scales reported beside the values (for error bounds): vscale2 = (1 / rho_i) sum_j m_j W_ij
 * |v_j - v_i|^2, gabs = (1 / rho_i) sum_j m_j |grad_i W_ij| |v_j - v_i|, gnorm = (1 / rho_i)
 * sum_j m_j |grad_i W_ij|, vmax = max over the neighbours of max_d |v_j,d|. */
typedef struct {
    int64_t j;
    double d[3]; /* r_i - r_j */
    double r;
} nbr_t;

typedef struct {
    nbr_t *e;
    int64_t n, cap;
} nbr_list;

static int nbr_push(nbr_list *L, int64_t j, const double d[3], double r)
{
    if (L->n == L->cap) {
        int64_t cap = L->cap ? 2 * L->cap : 256;
        nbr_t *e = (nbr_t *)realloc(L->e, (size_t)cap * sizeof(nbr_t));
        if (!e) return -1;
        L->e = e;
        L->cap = cap;
    }
    L->e[L->n].j = j;
    for (int k = 0; k < 3; k++) L->e[L->n].d[k] = d[k];
    L->e[L->n].r = r;
    L->n++;
    return 0;
}

/* Append j to the list when r_ij < h (the neighbour test of pair()). */
static int nbr_test(const pset *ps, int64_t i, int64_t j, double h2, nbr_list *L)
{
    const double *c[3] = {ps->x, ps->y, ps->z};
    double s[3]; /* r_j - r_i */
    for (int k = 0; k < 3; k++) {
        s[k] = c[k][j] - c[k][i];
        if (ps->periodic) s[k] = min_image(s[k], ps->box[k]);
    }
    double r2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
    if (r2 < h2) {
        const double d[3] = {-s[0], -s[1], -s[2]};
        return nbr_push(L, j, d, sqrt(r2));
    }
    return 0;
}

static int collect(const pset *ps, const bucket_grid *bg, int64_t i, double h, nbr_list *L)
{
    double h2 = h * h;
    L->n = 0;
    if (!bg) {
        for (int64_t j = 0; j < ps->n; j++)
            if (nbr_test(ps, i, j, h2, L)) return -1;
        return 0;
    }
    const double xi[3] = {ps->x[i], ps->y[i], ps->z[i]};
    int64_t lo[3], cnt[3];
    int64_t g = bg->g;
    bucket_box(ps, bg, xi, h, lo, cnt);
    for (int64_t kz = 0; kz < cnt[2]; kz++) {
        int64_t cz = lo[2] + kz;
        if (ps->periodic) cz = ((cz % g) + g) % g;
        for (int64_t ky = 0; ky < cnt[1]; ky++) {
            int64_t cy = lo[1] + ky;
            if (ps->periodic) cy = ((cy % g) + g) % g;
            for (int64_t kx = 0; kx < cnt[0]; kx++) {
                int64_t cx = lo[0] + kx;
                if (ps->periodic) cx = ((cx % g) + g) % g;
                int64_t id = cx + g * (cy + g * cz);
                int64_t s = lower_bound_id(bg->ids, ps->n, id);
                for (int64_t p = s; p < ps->n && bg->ids[p] == id; p++)
                    if (nbr_test(ps, i, bg->order[p], h2, L)) return -1;
            }
        }
    }
    return 0;
}

/* Velocity-field estimates of every target at its h (definitions above).  vel: three
 * arrays vx, vy, vz over all particles.  Outputs indexed by target position; vmean and
 * curl are three arrays of n_targets each (x block, y block, z block); scales holds
 * vscale2, gabs, gnorm, vmax in four blocks.  mode 0 = bucket grids, 1 = brute force. */
int oracle_interact(int64_t n, const double *x, const double *y, const double *z, const double *m,
                    const double *vx, const double *vy, const double *vz, const double *box,
                    int periodic, int64_t n_targets, const int64_t *targets, const double *h,
                    int mode, double *rho, double *vmean, double *sigma2, double *divv,
                    double *curlv, int64_t *count, double *scales, int kernel)
{
    const double pi = 3.14159265358979323846;
    pset ps;
    setup_pset(&ps, n, x, y, z, m, box, periodic, kernel);
    if (n_targets < 0) n_targets = n;
    const double sigma = kernel ? 1365.0 / (64.0 * pi) : 8.0 / pi;
    const double *v[3] = {vx, vy, vz};
    bucket_grid grids[ORACLE_MAX_LEVEL + 1];
    memset(grids, 0, sizeof(grids));
    if (mode == 0) {
        for (int64_t t = 0; t < n_targets; t++) {
            int k = level_for(&ps, h[t]);
            if (!grids[k].built && build_grid(&ps, k, &grids[k]) != 0) return -1;
        }
    }
    int failed = 0;
    #pragma omp parallel
    {
        nbr_list L = {NULL, 0, 0};
        #pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < n_targets; t++) {
            const int64_t i = targets ? targets[t] : t;
            const double hi = h[t];
            if (collect(&ps, mode == 0 ? &grids[level_for(&ps, hi)] : NULL, i, hi, &L)) {
                #pragma omp atomic write
                failed = 1;
                continue;
            }
            /* density, Eq. (1) */
            double r_sum = 0.0;
            for (int64_t k = 0; k < L.n; k++) {
                double q = L.e[k].r / hi;
                double w = kernel ? oracle_w_c6(q) : oracle_w(q);
                double W = sigma / (hi * hi * hi) * w;
                r_sum += ps.m[L.e[k].j] * W;
            }
            const double rh = r_sum;
            /* kernel-weighted mean velocity */
            double vb[3] = {0.0, 0.0, 0.0};
            for (int64_t k = 0; k < L.n; k++) {
                const int64_t j = L.e[k].j;
                double q = L.e[k].r / hi;
                double w = kernel ? oracle_w_c6(q) : oracle_w(q);
                double W = sigma / (hi * hi * hi) * w;
                for (int d = 0; d < 3; d++) vb[d] += ps.m[j] * W * v[d][j];
            }
            for (int d = 0; d < 3; d++) vb[d] = vb[d] / rh;
            /* dispersion about the mean; divergence and curl; the scales */
            double s2 = 0.0, dv_sum = 0.0, cv[3] = {0.0, 0.0, 0.0};
            double vs2 = 0.0, gabs = 0.0, gnorm = 0.0, vmax = 0.0;
            for (int64_t k = 0; k < L.n; k++) {
                const int64_t j = L.e[k].j;
                const double r = L.e[k].r;
                double q = r / hi;
                double w = kernel ? oracle_w_c6(q) : oracle_w(q);
                double W = sigma / (hi * hi * hi) * w;
                double e[3], dvel[3];
                for (int d = 0; d < 3; d++) {
                    e[d] = v[d][j] - vb[d];
                    dvel[d] = v[d][j] - v[d][i];
                    if (fabs(v[d][j]) > vmax) vmax = fabs(v[d][j]);
                }
                s2 += ps.m[j] * W * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
                vs2 += ps.m[j] * W * (dvel[0] * dvel[0] + dvel[1] * dvel[1] + dvel[2] * dvel[2]);
                /* grad_i W_ij = dW/dr (r_i - r_j) / r, zero at r = 0 */
                double gW[3] = {0.0, 0.0, 0.0};
                if (r > 0.0) {
                    double wp = -(kernel ? oracle_mqdw_c6(q) : oracle_mqdw(q)) / q;
                    double dWdr = sigma / (hi * hi * hi * hi) * wp;
                    for (int d = 0; d < 3; d++) gW[d] = dWdr * (L.e[k].d[d] / r);
                }
                dv_sum += ps.m[j] * (dvel[0] * gW[0] + dvel[1] * gW[1] + dvel[2] * gW[2]);
                /* (v_i - v_j) x grad_i W */
                const double u[3] = {-dvel[0], -dvel[1], -dvel[2]};
                cv[0] += ps.m[j] * (u[1] * gW[2] - u[2] * gW[1]);
                cv[1] += ps.m[j] * (u[2] * gW[0] - u[0] * gW[2]);
                cv[2] += ps.m[j] * (u[0] * gW[1] - u[1] * gW[0]);
                double gn = sqrt(gW[0] * gW[0] + gW[1] * gW[1] + gW[2] * gW[2]);
                gnorm += ps.m[j] * gn;
                gabs += ps.m[j] * gn * sqrt(dvel[0] * dvel[0] + dvel[1] * dvel[1] + dvel[2] * dvel[2]);
            }
            rho[t] = rh;
            for (int d = 0; d < 3; d++) {
                vmean[d * n_targets + t] = vb[d];
                curlv[d * n_targets + t] = cv[d] / rh;
            }
            sigma2[t] = s2 / rh;
            divv[t] = dv_sum / rh;
            count[t] = L.n;
            scales[t] = vs2 / rh;
            scales[n_targets + t] = gabs / rh;
            scales[2 * n_targets + t] = gnorm / rh;
            scales[3 * n_targets + t] = vmax;
        }
        free(L.e);
    }
    for (int k = 0; k <= ORACLE_MAX_LEVEL; k++)
        if (grids[k].built) free_grid(&grids[k]);
    return failed ? -1 : 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
