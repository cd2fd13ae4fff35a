// sph_capi.cu -- the C ABI (include/sph.h): context, one-time scratch arena, argument
// checks, and the host orchestration of sort -> pass loop -> scatter on the context's
// stream.  No CUDA type crosses the ABI; every failure becomes an sph_status plus a
// per-context message.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "sph.h"
#include "sph_kernels.cuh"

using namespace sph;

struct sph_ctx {
    sph_params params{};
    std::string tune_cache;
    int64_t capacity = 0;
    int64_t max_groups = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    std::string gpu_name;
    std::string last_error;

    // sorted state
    bool sorted = false;
    bool fp64_records = false;  // the sort filled the FP64 records (an FP64 sort)
    int64_t n = 0;
    KeyLayout kl{};
    int which = 0;  // key/idx buffer holding the sorted order
    SegInfo seg_host{};

    // device arena
    void *arena = nullptr;
    uint64_t *key[2] = {nullptr, nullptr};
    int32_t *idx[2] = {nullptr, nullptr};
    int32_t *hist = nullptr, *hist_off = nullptr, *scan_aux = nullptr;
    uint4 *pfix = nullptr;
    double4_32a *pdbl = nullptr;
    int32_t *ctab = nullptr;
    SegInfo *segs = nullptr;
    double *h = nullptr, *hlo = nullptr, *hhi = nullptr, *e_h = nullptr, *e_rho = nullptr,
           *e_nw = nullptr, *e_dnw = nullptr;
    int32_t *e_cnt = nullptr, *todo[2] = {nullptr, nullptr}, *flags = nullptr, *items = nullptr;
    int32_t *tsize = nullptr, *toff = nullptr;
    int32_t *nb_slot = nullptr;  // neighbour export: caller index -> sample row
    int32_t *lst = nullptr, *lst_n = nullptr, *todo_s = nullptr;  // cached neighbour lists
    double *lst_r = nullptr;
    void *vrec = nullptr;  // sorted velocities of the interaction pass (32 bytes a particle)
    float *h32 = nullptr, *e_rho32 = nullptr, *e_nw32 = nullptr, *e_dnw32 = nullptr;
    DevState *ds = nullptr;

    // pinned host mirrors
    DevState *ds_host = nullptr;
    SegInfo *seg_pinned = nullptr;
    int64_t *i64_pinned = nullptr;

    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t dev_ev[2 * SPH_MAX_PASSES] = {};  // around each density launch

    // CUDA graph of the pass loop (a conditional while node whose body runs two passes)
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture the body
    cudaGraph_t loop_graph = nullptr;
    cudaGraphExec_t loop_exec = nullptr;
    int body_kernels = 0;               // kernels per body execution
    struct {
        int64_t n = -1;
        int which = -1, precision = -1, grid = -1;
        sph_tuning tuning{};
        KeyLayout kl{};
    } graph_key;
    sph_tuning tuning{0, 3, 1, 0, 0, 32, 256, 0, 10, 0, 0};
    int launches = 0;
    int sort_launches = 0;  // kernels of the last sort stage
    int grid_cap = 0;
    // resident density blocks per SM: [FP64, FP32 with queue, FP32 direct][64, 128, 256 threads]
    // (0 = not asked yet)
    int occupancy[3][3] = {};
};

namespace {

constexpr int64_t kMaxCapacity = (1ll << 31) - (1ll << 20);
constexpr int64_t kMaxGroupsCap = 1ll << 20;

sph_status fail(sph_ctx *c, sph_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return s;
}

sph_status cuda_fail(sph_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, SPH_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CU(ctx, expr, where)                                                                  \
    do {                                                                                      \
        cudaError_t e__ = (expr);                                                             \
        if (e__ != cudaSuccess) return cuda_fail((ctx), e__, (where));                        \
    } while (0)

sph_status check_params(sph_ctx *c, const sph_params *p)
{
    if (!p) return fail(c, SPH_ERR_INVALID_ARG, "params is NULL");
    if (p->kernel != SPH_KERNEL_M4 && p->kernel != SPH_KERNEL_WENDLAND_C6)
        return fail(c, SPH_ERR_INVALID_ARG, "unknown kernel %d", p->kernel);
    const double self = p->kernel == SPH_KERNEL_M4 ? 32.0 / 3.0 : 1365.0 / 48.0;
    if (p->precision != SPH_PREC_FP64 && p->precision != SPH_PREC_FP32_KAHAN)
        return fail(c, SPH_ERR_INVALID_ARG, "unknown precision %d", p->precision);
    if (p->periodic != 0 && p->periodic != 1) return fail(c, SPH_ERR_INVALID_ARG, "periodic must be 0 or 1");
    if (p->periodic)
        for (int d = 0; d < 3; d++)
            if (!(p->box[d] > 0.0 && p->box[d] <= DBL_MAX))
                return fail(c, SPH_ERR_INVALID_ARG, "box[%d] must be finite and > 0", d);
    if (!(p->nngb > self && p->nngb <= 1e9))
        return fail(c, SPH_ERR_INVALID_ARG, "nngb must exceed the self term %g (got %g)", self, p->nngb);
    if (!(p->tol >= 0.0 && p->tol <= DBL_MAX)) return fail(c, SPH_ERR_INVALID_ARG, "tol must be >= 0");
    if (p->max_iter < 1 || p->max_iter > SPH_MAX_PASSES)
        return fail(c, SPH_ERR_INVALID_ARG, "max_iter must be in [1, %d]", SPH_MAX_PASSES);
    if (p->use_graph != 0 && p->use_graph != 1) return fail(c, SPH_ERR_INVALID_ARG, "use_graph must be 0 or 1");
    if (p->list_entries != 0 && (p->list_entries < 16 || p->list_entries > 1024))
        return fail(c, SPH_ERR_INVALID_ARG, "list_entries must be 0 or in [16, 1024]");
    return SPH_OK;
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// Carve every buffer out of one allocation; with base == nullptr only the size is computed.
size_t carve(sph_ctx *c, char *base)
{
    const int64_t cap = c->capacity;
    const int64_t hs = radix_hist_size(cap);
    const int64_t aux = scan_aux_size(std::max<int64_t>(cap, hs)) + 8;
    // periodic: 8^lc + 1 <= 8 n + 1 entries (one extra table level at most); batch groups:
    // sum of (8^lc + 1) <= 8 n + groups
    const int64_t ctab_cap = 8 * cap + c->max_groups + 2;
    const int64_t gcap = c->max_groups;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        void *p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    for (int k = 0; k < 2; k++) c->key[k] = (uint64_t *)take(cap * 8);
    for (int k = 0; k < 2; k++) c->idx[k] = (int32_t *)take(cap * 4);
    c->hist = (int32_t *)take(hs * 4);
    c->hist_off = (int32_t *)take(hs * 4);
    c->scan_aux = (int32_t *)take(aux * 4);
    c->pfix = (uint4 *)take(cap * 16);
    c->pdbl = (double4_32a *)take(cap * 32);
    c->ctab = (int32_t *)take(ctab_cap * 4);
    c->segs = (SegInfo *)take((gcap + 1) * sizeof(SegInfo));
    c->h = (double *)take(cap * 8);
    c->hlo = (double *)take(cap * 8);
    c->hhi = (double *)take(cap * 8);
    c->e_h = (double *)take(cap * 8);
    c->e_rho = (double *)take(cap * 8);
    c->e_nw = (double *)take(cap * 8);
    c->e_dnw = (double *)take(cap * 8);
    c->e_cnt = (int32_t *)take(cap * 4);
    for (int k = 0; k < 2; k++) c->todo[k] = (int32_t *)take(cap * 4);
    c->flags = (int32_t *)take(cap * 4);
    c->items = (int32_t *)take((cap + 1) * 4);
    c->h32 = (float *)take(cap * 4);
    c->e_rho32 = (float *)take(cap * 4);
    c->e_nw32 = (float *)take(cap * 4);
    c->e_dnw32 = (float *)take(cap * 4);
    c->tsize = (int32_t *)take((gcap + 1) * 4);
    c->toff = (int32_t *)take((gcap + 1) * 4);
    c->nb_slot = (int32_t *)take(cap * 4);
    const int64_t le = c->params.list_entries;
    c->lst = le > 0 ? (int32_t *)take((size_t)cap * (size_t)le * 4) : nullptr;
    c->lst_n = le > 0 ? (int32_t *)take(cap * 4) : nullptr;
    c->lst_r = le > 0 ? (double *)take(cap * 8) : nullptr;
    c->todo_s = le > 0 ? (int32_t *)take(cap * 4) : nullptr;
    c->vrec = take((size_t)cap * 32);
    c->ds = (DevState *)take(sizeof(DevState));
    return off;
}

SortArgs sort_args(sph_ctx *c)
{
    SortArgs a{};
    for (int k = 0; k < 2; k++) {
        a.key[k] = c->key[k];
        a.idx[k] = c->idx[k];
    }
    a.hist = c->hist;
    a.hist_off = c->hist_off;
    a.scan_aux = c->scan_aux;
    a.pfix = c->pfix;
    a.pdbl = c->pdbl;
    a.ctab = c->ctab;
    a.segs = c->segs;
    a.ds = c->ds;
    a.kl = c->kl;
    a.grid_cap = c->grid_cap;
    a.table_extra = c->tuning.table_extra;
    a.self_floor = c->params.kernel == SPH_KERNEL_WENDLAND_C6 ? 1365.0 / 48.0 : 32.0 / 3.0;
    a.launches = &c->launches;
    return a;
}

SolveArgs solve_args(sph_ctx *c)
{
    SolveArgs a{};
    a.pfix = c->pfix;
    a.pdbl = c->pdbl;
    a.key = c->key[c->which];
    a.idx = c->idx[c->which];
    a.segs = c->segs;
    a.ctab = c->ctab;
    a.kl = c->kl;
    a.n = c->n;
    a.h = c->h;
    a.hlo = c->hlo;
    a.hhi = c->hhi;
    a.e_h = c->e_h;
    a.e_rho = c->e_rho;
    a.e_nw = c->e_nw;
    a.e_dnw = c->e_dnw;
    a.e_cnt = c->e_cnt;
    a.h32 = c->h32;
    a.e_rho32 = c->e_rho32;
    a.e_nw32 = c->e_nw32;
    a.e_dnw32 = c->e_dnw32;
    a.todo[0] = c->todo[0];
    a.todo[1] = c->todo[1];
    a.flags = c->flags;
    a.items = c->items;
    a.scan_aux = c->scan_aux;
    a.ds = c->ds;
    a.grid_cap = c->grid_cap;
    a.precision = c->params.precision;
    a.kernel = c->params.kernel;
    {
        const int mode = c->params.precision == SPH_PREC_FP64 ? 0 : c->tuning.direct_pct == 0 ? 2 : 1;
        const int bt = c->tuning.block_threads;
        const int ti = bt == 64 ? 0 : bt == 128 ? 1 : 2;
        int &occ = c->occupancy[mode][ti];
        if (occ == 0) occ = density_blocks_per_sm(c->params.precision, c->tuning.direct_pct, bt);
        const int bps = c->tuning.blocks_per_sm > 0 && c->tuning.blocks_per_sm < occ ? c->tuning.blocks_per_sm : occ;
        a.density_grid = c->num_sms * bps;
        a.block_threads = bt;
    }
    a.gmax = c->tuning.item_max;
    a.gmax_sparse = c->tuning.sparse_item_max > 0 ? c->tuning.sparse_item_max : c->tuning.item_max;
    a.item_cap = c->tuning.item_cap;
    // cached neighbour lists (the FP32 per-lane queue of direct_pct > 0 records none)
    const bool lists = c->params.list_entries > 0 && (c->params.precision == SPH_PREC_FP64 || c->tuning.direct_pct == 0);
    a.lst = lists ? c->lst : nullptr;
    a.lst_n = c->lst_n;
    a.lst_r = c->lst_r;
    a.todo_s = c->todo_s;
    a.list_entries = c->params.list_entries;
    a.list_margin = 1.0f + (float)c->tuning.list_margin_pct * 0.01f;
    a.group_shift = c->tuning.group_shift;
    a.sparse_shift = c->tuning.sparse_shift;
    a.cell_div = c->tuning.cell_div;
    a.direct_pct = c->tuning.direct_pct;
    a.free_first = (c->kl.seg_bits == 0 && c->params.precision != SPH_PREC_FP64 &&
                    c->tuning.direct_pct == 0) ? 1 : 0;
    a.cubic = (c->seg_host.q[0] == c->seg_host.q[1] && c->seg_host.q[1] == c->seg_host.q[2]) ? 1 : 0;
    a.launches = &c->launches;
    return a;
}

// Level of the dense cell table: the finest level with at most 8^extra cells per particle.
int table_level(int64_t n, int lmax, int extra)
{
    int lc = 0;
    while (lc < lmax && lc < 10 && (1ll << (3 * (lc + 1))) <= (n << (3 * extra))) lc++;
    return lc;
}

// Autotuner cache: one line per result,
// "<gpu>|<log2 n>|<periodic>|<precision> gs cd te dp ic im bt bs lm ss sm" (the sph_tuning
// fields in order; a line without the last field leaves it at its default); the last matching
// line wins.
std::string cache_key(const sph_ctx *c, int64_t n)
{
    int b = 0;
    while ((2ll << b) <= n) b++;
    char buf[256];
    snprintf(buf, sizeof(buf), "%s|%d|%d|%d", c->gpu_name.c_str(), b, c->params.periodic, c->params.precision);
    return buf;
}

bool cache_lookup(const sph_ctx *c, int64_t n, sph_tuning *t)
{
    if (c->tune_cache.empty()) return false;
    FILE *f = fopen(c->tune_cache.c_str(), "r");
    if (!f) return false;
    const std::string key = cache_key(c, n);
    char line[512], k[300];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        sph_tuning x = c->tuning;
        x.sparse_item_max = 0;
        const int got = sscanf(line, "%299s %d %d %d %d %d %d %d %d %d %d %d", k, &x.group_shift, &x.cell_div,
                               &x.table_extra, &x.direct_pct, &x.item_cap, &x.item_max, &x.block_threads,
                               &x.blocks_per_sm, &x.list_margin_pct, &x.sparse_shift, &x.sparse_item_max);
        if ((got == 11 || got == 12) && key == k) {
            *t = x;
            found = true;
        }
    }
    fclose(f);
    return found;
}

void cache_store(const sph_ctx *c, int64_t n, const sph_tuning &t)
{
    if (c->tune_cache.empty()) return;
    FILE *f = fopen(c->tune_cache.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d %d\n", cache_key(c, n).c_str(), t.group_shift, t.cell_div,
            t.table_extra, t.direct_pct, t.item_cap, t.item_max, t.block_threads, t.blocks_per_sm,
            t.list_margin_pct, t.sparse_shift, t.sparse_item_max);
    fclose(f);
}

bool tuning_ok(const sph_tuning *t)
{
    const bool pow2 = t && t->item_max >= 1 && t->item_max <= 32 && (t->item_max & (t->item_max - 1)) == 0;
    return t && t->group_shift >= -2 && t->group_shift <= 3 && t->cell_div >= 1 && t->cell_div <= 3 &&
           t->table_extra >= 0 && t->table_extra <= 1 && t->direct_pct >= 0 && t->direct_pct <= 101 &&
           (t->item_cap == 0 || (t->item_cap >= 2 && t->item_cap <= 64)) && pow2 &&
           (t->block_threads == 64 || t->block_threads == 128 || t->block_threads == 256) &&
           t->blocks_per_sm >= 0 && t->blocks_per_sm <= 32 && t->list_margin_pct >= 1 && t->list_margin_pct <= 100 &&
           t->sparse_shift >= -2 && t->sparse_shift <= 3 &&
           (t->sparse_item_max == 0 ||
            (t->sparse_item_max <= 32 && (t->sparse_item_max & (t->sparse_item_max - 1)) == 0));
}

sph_status read_state(sph_ctx *c)
{
    CU(c, cudaMemcpyAsync(c->ds_host, c->ds, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream),
       "reading the device state");
    CU(c, cudaStreamSynchronize(c->stream), "synchronising the stream");
    return SPH_OK;
}

sph_status device_status_error(sph_ctx *c, int bits)
{
    std::string what;
    if (bits & kBadPosition) what += " non-finite or out-of-box position;";
    if (bits & kBadMass) what += " non-positive or non-finite mass;";
    if (bits & kBadH) what += " h not in (0, min(box)/2) or bad group nngb/tol;";
    if (bits & 8) what += " internal cell-count guard;";
    if (bits & kBadSample) what += " sample index outside [0, n) or repeated;";
    if (bits & kBadVelocity) what += " non-finite velocity;";
    return fail(c, SPH_ERR_DEVICE_STATUS, "device flagged the input:%s", what.c_str());
}

void drop_graph(sph_ctx *c)
{
    if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
    if (c->loop_graph) cudaGraphDestroy(c->loop_graph);
    c->loop_exec = nullptr;
    c->loop_graph = nullptr;
    c->graph_key.n = -1;
}

// Executable graph of the pass loop: a conditional while node whose body runs two passes
// (todo list 0 -> 1, then 1 -> 0) and sets the loop condition on the device, so the loop
// needs no host round trip per pass.  Rebuilt only when the launch arguments change.
sph_status loop_graph(sph_ctx *c, const SolveArgs &a0)
{
    const bool same = c->graph_key.n == c->n && c->graph_key.which == c->which &&
                      c->graph_key.precision == a0.precision && c->graph_key.grid == a0.density_grid &&
                      memcmp(&c->graph_key.tuning, &c->tuning, sizeof(sph_tuning)) == 0 &&
                      memcmp(&c->graph_key.kl, &c->kl, sizeof(KeyLayout)) == 0 && c->loop_exec;
    if (same) return SPH_OK;
    drop_graph(c);
    SolveArgs a = a0;
    a.dens_ev[0] = a.dens_ev[1] = nullptr;
    int launches = 0;
    a.launches = &launches;
    cudaGraph_t g = nullptr;
    CU(c, cudaGraphCreate(&g, 0), "creating the loop graph");
    c->loop_graph = g;
    cudaGraphConditionalHandle handle;
    CU(c, cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault), "loop condition");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = handle;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CU(c, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p), "conditional node");
    cudaGraph_t body = p.conditional.phGraph_out[0];
    CU(c, cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal),
       "capturing the loop body");
    cudaError_t e1 = launch_pass(a, 0, true, c->cap_stream);
    cudaError_t e2 = launch_pass(a, 1, true, c->cap_stream);
    cudaError_t e3 = launch_set_loop(handle, c->ds, c->cap_stream);
    cudaError_t e4 = cudaStreamEndCapture(c->cap_stream, &body);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
        cudaGetLastError();
        drop_graph(c);
        return cuda_fail(c, e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4,
                         "capturing the loop body");
    }
    CU(c, cudaGraphInstantiate(&c->loop_exec, g, 0), "instantiating the loop graph");
    c->body_kernels = launches + 1;
    c->graph_key.n = c->n;
    c->graph_key.which = c->which;
    c->graph_key.precision = a0.precision;
    c->graph_key.grid = a0.density_grid;
    c->graph_key.tuning = c->tuning;
    c->graph_key.kl = c->kl;
    return SPH_OK;
}

// Host-driven pass loop (one todo-count read per pass); returns the passes run.
sph_status host_passes(sph_ctx *c, SolveArgs &a, bool events, int *passes_run)
{
    cudaStream_t st = c->stream;
    int cur = 0;
    *passes_run = 0;
    for (int pass = 0; pass < c->params.max_iter; pass++) {
        a.dens_ev[0] = events ? c->dev_ev[2 * pass] : nullptr;
        a.dens_ev[1] = events ? c->dev_ev[2 * pass + 1] : nullptr;
        CU(c, launch_pass(a, cur, true, st), "density pass");
        *passes_run = pass + 1;
        CU(c, cudaMemcpyAsync(&c->ds_host->todo_count, &c->ds->todo_count, sizeof(int32_t),
                              cudaMemcpyDeviceToHost, st),
           "reading the todo count");
        CU(c, cudaStreamSynchronize(st), "synchronising the pass");
        cur = 1 - cur;
        if (c->ds_host->todo_count == 0) break;
    }
    return SPH_OK;
}

// The pass loop shared by sph_density_solve and sph_batch_solve.
sph_status run_solve(sph_ctx *c, double *h_inout, double *rho_out, int32_t *count_out,
                     double *nw_out, sph_stats *stats)
{
    cudaStream_t st = c->stream;
    const bool graph = c->params.use_graph != 0;
    const int launches0 = c->launches;
    SolveArgs a = solve_args(c);
    sph_status s = SPH_OK;
    if (graph) {
        s = loop_graph(c, a);
        if (s != SPH_OK) return s;
    }
    CU(c, cudaEventRecord(c->ev[2], st), "event");
    CU(c, cudaMemsetAsync(&c->ds->status, 0, sizeof(int32_t), st), "clearing the status word");
    CU(c, cudaMemsetAsync(&c->ds->h_varies, 0, sizeof(int32_t), st), "clearing the h flag");
    CU(c, launch_solve_init(a, h_inout, c->params.max_iter, st), "solve init");
    if (!graph) {
        s = read_state(c);
        if (s != SPH_OK) return s;
        if (c->ds_host->status | c->ds_host->sort_status)
            return device_status_error(c, c->ds_host->status | c->ds_host->sort_status);
    }

    int passes_run = 0;
    if (graph) {
        CU(c, cudaGraphLaunch(c->loop_exec, st), "launching the loop graph");
    } else {
        s = host_passes(c, a, true, &passes_run);
        if (s != SPH_OK) return s;
    }
    CU(c, launch_scatter(a, h_inout, rho_out, count_out, nw_out, nullptr, st), "scatter");
    CU(c, cudaEventRecord(c->ev[3], st), "event");
    s = read_state(c);
    if (s != SPH_OK) return s;
    const DevState &d = *c->ds_host;
    // the while body (two passes) ran ceil(passes / 2) times
    if (graph) c->launches += (d.pass > 0 ? (d.pass + 1) / 2 : 1) * c->body_kernels;
    if (d.status | d.sort_status) return device_status_error(c, d.status | d.sort_status);
    if (stats) {
        stats->passes = d.pass;
        stats->kernel_launches = c->launches - launches0 + c->sort_launches;
        for (int k = 0; k < SPH_MAX_PASSES; k++) stats->todo_per_pass[k] = k < d.pass ? d.todo_per_pass[k] : 0;
        stats->unconverged = d.todo_count;
        stats->exceeded = d.exceeded;
        stats->pair_evals = (int64_t)d.pair_evals;
        stats->pair_tests = (int64_t)d.pair_tests;
        stats->list_evals = (int64_t)d.list_evals;
        for (int k = 0; k < SPH_MAX_PASSES; k++)
            stats->pairs_per_pass[k] = k < d.pass ? (int64_t)d.pairs_per_pass[k] : 0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]);
        stats->solve_ms = ms;
        double dms = 0.0;
        for (int k = 0; k < passes_run; k++) {
            float m = 0.f;
            if (cudaEventElapsedTime(&m, c->dev_ev[2 * k], c->dev_ev[2 * k + 1]) == cudaSuccess) {
                dms += m;
                stats->density_ms_per_pass[k] = m;
            }
        }
        stats->density_ms = dms;
        stats->density_launches = passes_run;
    }
    if (d.exceeded > 0)
        return fail(c, SPH_ERR_H_EXCEEDS_BOX, "%d particles needed h >= min(box)/2", d.exceeded);
    if (d.todo_count > 0)
        return fail(c, SPH_ERR_NOT_CONVERGED, "%d particles unconverged after %d passes", d.todo_count,
                    d.pass);
    return SPH_OK;
}

}  // namespace

extern "C" {

const char *sph_status_string(sph_status s)
{
    switch (s) {
    case SPH_OK: return "ok";
    case SPH_ERR_INVALID_ARG: return "invalid argument";
    case SPH_ERR_CUDA: return "CUDA error";
    case SPH_ERR_OOM: return "capacity exceeded or device allocation failed";
    case SPH_ERR_NOT_SORTED: return "sph_sort must run first";
    case SPH_ERR_H_EXCEEDS_BOX: return "h reached half the periodic box";
    case SPH_ERR_NOT_CONVERGED: return "not converged within max_iter passes";
    case SPH_ERR_DEVICE_STATUS: return "the device flagged invalid input";
    case SPH_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

const char *sph_last_error(const sph_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

sph_status sph_create(const sph_params *params, int64_t capacity, void *cuda_stream, sph_ctx **out)
{
    if (!out) return SPH_ERR_INVALID_ARG;
    *out = nullptr;
    sph_status s = check_params(nullptr, params);
    if (s != SPH_OK) return s;
    if (capacity < 1 || capacity > kMaxCapacity) return SPH_ERR_INVALID_ARG;
    sph_ctx *c = new (std::nothrow) sph_ctx();
    if (!c) return SPH_ERR_OOM;
    c->params = *params;
    if (params->tune_cache) c->tune_cache = params->tune_cache;
    c->params.tune_cache = nullptr;
    c->capacity = capacity;
    c->max_groups = std::min<int64_t>(capacity, kMaxGroupsCap);
    c->stream = (cudaStream_t)cuda_stream;
    auto bail = [&](sph_status st) {
        sph_destroy(c);
        return st;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(SPH_ERR_CUDA);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(SPH_ERR_CUDA);
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return bail(SPH_ERR_CUDA);
        c->gpu_name = prop.name;
        for (char &ch : c->gpu_name)
            if (ch == ' ' || ch == '|') ch = '_';
    }
    const size_t bytes = carve(c, nullptr);
    if (cudaMalloc(&c->arena, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->arena = nullptr;
        return bail(SPH_ERR_OOM);
    }
    carve(c, (char *)c->arena);
    if (cudaMallocHost((void **)&c->ds_host, sizeof(DevState)) != cudaSuccess ||
        cudaMallocHost((void **)&c->seg_pinned, sizeof(SegInfo)) != cudaSuccess ||
        cudaMallocHost((void **)&c->i64_pinned, 2 * sizeof(int64_t)) != cudaSuccess)
        return bail(SPH_ERR_OOM);
    for (int k = 0; k < 4; k++)
        if (cudaEventCreate(&c->ev[k]) != cudaSuccess) return bail(SPH_ERR_CUDA);
    for (int k = 0; k < 2 * SPH_MAX_PASSES; k++)
        if (cudaEventCreate(&c->dev_ev[k]) != cudaSuccess) return bail(SPH_ERR_CUDA);
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(SPH_ERR_CUDA);
    c->grid_cap = c->num_sms * 16;
    if (cudaMemset(c->ds, 0, sizeof(DevState)) != cudaSuccess) return bail(SPH_ERR_CUDA);
    *out = c;
    return SPH_OK;
}

sph_status sph_get_tuning(const sph_ctx *ctx, sph_tuning *out)
{
    if (!ctx || !out) return SPH_ERR_INVALID_ARG;
    *out = ctx->tuning;
    return SPH_OK;
}

sph_status sph_set_tuning(sph_ctx *ctx, const sph_tuning *tuning)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!tuning_ok(tuning)) return fail(ctx, SPH_ERR_INVALID_ARG, "tuning value out of range");
    if (tuning->table_extra != ctx->tuning.table_extra) ctx->sorted = false;
    ctx->tuning = *tuning;
    return SPH_OK;
}

sph_status sph_set_params(sph_ctx *ctx, const sph_params *params)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    sph_status s = check_params(ctx, params);
    if (s != SPH_OK) return s;
    if (params->list_entries != ctx->params.list_entries)
        return fail(ctx, SPH_ERR_INVALID_ARG, "list_entries is fixed when the context is created");
    const bool geometry_changed = params->periodic != ctx->params.periodic ||
                                  params->box[0] != ctx->params.box[0] ||
                                  params->box[1] != ctx->params.box[1] ||
                                  params->box[2] != ctx->params.box[2] ||
                                  // an FP32 sort keeps no FP64 records
                                  (params->precision == SPH_PREC_FP64 && !ctx->fp64_records);
    ctx->params = *params;
    ctx->tune_cache = params->tune_cache ? params->tune_cache : "";
    ctx->params.tune_cache = nullptr;
    if (geometry_changed) ctx->sorted = false;
    return SPH_OK;
}

void sph_destroy(sph_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream || ctx->arena) cudaStreamSynchronize(ctx->stream);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->ds_host) cudaFreeHost(ctx->ds_host);
    if (ctx->seg_pinned) cudaFreeHost(ctx->seg_pinned);
    if (ctx->i64_pinned) cudaFreeHost(ctx->i64_pinned);
    for (int k = 0; k < 4; k++)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    for (int k = 0; k < 2 * SPH_MAX_PASSES; k++)
        if (ctx->dev_ev[k]) cudaEventDestroy(ctx->dev_ev[k]);
    drop_graph(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

sph_status sph_sort(sph_ctx *ctx, int64_t n, const double *pos_xyz_dev, const double *mass_dev)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    ctx->sorted = false;
    if (!pos_xyz_dev || !mass_dev) return fail(ctx, SPH_ERR_INVALID_ARG, "NULL position or mass pointer");
    if (n < 1) return fail(ctx, SPH_ERR_INVALID_ARG, "n must be >= 1 (got %lld)", (long long)n);
    if (n > ctx->capacity)
        return fail(ctx, SPH_ERR_OOM, "n = %lld exceeds the context capacity %lld", (long long)n,
                    (long long)ctx->capacity);
    if (!ctx->params.periodic)
        return fail(ctx, SPH_ERR_UNSUPPORTED, "sph_sort needs periodic = 1; open particle sets go "
                                              "through sph_batch_solve (one group per set)");
    cudaStream_t st = ctx->stream;
    const sph_params &p = ctx->params;
    {
        sph_tuning cached;
        if (cache_lookup(ctx, n, &cached) && tuning_ok(&cached)) ctx->tuning = cached;
    }
    ctx->n = n;
    // 16 octree levels (cells down to 2^-16 of the box) in 48-bit keys: six radix passes.  The
    // grouping and enumeration levels never go finer than the key (only a cell's candidate count,
    // not the result, depends on it), and no work item needs cells that fine unless h is below
    // about 1e-5 of the box.
    ctx->kl.lmax = 16;
    ctx->kl.seg_bits = 0;
    ctx->kl.key_bits = 48;
    ctx->kl.coord_bits = 32;
    SegInfo &sg = ctx->seg_host;
    memset(&sg, 0, sizeof(sg));
    for (int d = 0; d < 3; d++) {
        sg.q[d] = std::ldexp(p.box[d], -32);      // exact: a power-of-two scaling
        sg.inv_q[d] = std::ldexp(1.0 / p.box[d], 32);
        sg.origin[d] = 0.0;
        sg.box[d] = p.box[d];
    }
    sg.nngb = p.nngb;
    sg.tol = p.tol;
    sg.half_box = 0.5 * std::min(p.box[0], std::min(p.box[1], p.box[2]));
    sg.periodic = 1;
    sg.level_c = table_level(n, ctx->kl.lmax, ctx->tuning.table_extra);
    sg.tab_off = 0;
    sg.start = 0;
    sg.end = (int32_t)n;
    *ctx->seg_pinned = sg;
    CU(ctx, cudaEventRecord(ctx->ev[0], st), "event");
    CU(ctx, cudaMemcpyAsync(ctx->segs, ctx->seg_pinned, sizeof(SegInfo), cudaMemcpyHostToDevice, st),
       "uploading the segment");
    CU(ctx, cudaMemsetAsync(ctx->ds, 0, sizeof(DevState), st), "clearing the device state");
    const int launches0 = ctx->launches;
    SortArgs a = sort_args(ctx);
    // FP32 solves read only the fixed-point records: the key kernel leaves them in caller order in
    // the FP64 records' memory and the gather moves one record per particle; an FP64 sort gathers
    // both from the caller's arrays
    const bool fp64 = p.precision == SPH_PREC_FP64;
    uint4 *rec = fp64 ? nullptr : (uint4 *)ctx->pdbl;
    CU(ctx, launch_keys_periodic(a, n, pos_xyz_dev, mass_dev, sg, p.box, st, rec), "morton keys");
    int which = 0;
    CU(ctx, launch_radix_sort(a, n, &which, st), "radix sort");
    ctx->which = which;
    if (fp64)
        CU(ctx, launch_gather_periodic(a, n, pos_xyz_dev, mass_dev, ctx->idx[which], sg, st), "gather");
    else
        CU(ctx, launch_gather_rec(a, n, ctx->idx[which], rec, st), "gather");
    ctx->fp64_records = fp64;
    CU(ctx, launch_cell_table(a, n, ctx->key[which], st), "cell table");
    CU(ctx, cudaEventRecord(ctx->ev[1], st), "event");
    ctx->sort_launches = ctx->launches - launches0;
    if (!ctx->params.use_graph) {
        // without graphs the sort reports bad input itself; with graphs it stays
        // asynchronous and the solve reports it
        sph_status s = read_state(ctx);
        if (s != SPH_OK) return s;
        if (ctx->ds_host->sort_status) return device_status_error(ctx, ctx->ds_host->sort_status);
    }
    ctx->sorted = true;
    return SPH_OK;
}

sph_status sph_density_solve(sph_ctx *ctx, double *h_inout_dev, double *rho_out_dev,
                             int32_t *count_out_dev, double *nw_out_dev, sph_stats *stats)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!h_inout_dev || !rho_out_dev || !count_out_dev)
        return fail(ctx, SPH_ERR_INVALID_ARG, "NULL h, rho or count pointer");
    if (!ctx->sorted) return fail(ctx, SPH_ERR_NOT_SORTED, "sph_sort has not run on this context");
    if (stats) memset(stats, 0, sizeof(*stats));
    // the band and pass limit may have changed since the sort
    SegInfo sg = ctx->seg_host;
    sg.nngb = ctx->params.nngb;
    sg.tol = ctx->params.tol;
    *ctx->seg_pinned = sg;
    CU(ctx, cudaMemcpyAsync(ctx->segs, ctx->seg_pinned, sizeof(SegInfo), cudaMemcpyHostToDevice,
                            ctx->stream),
       "uploading the segment");
    sph_status s = run_solve(ctx, h_inout_dev, rho_out_dev, count_out_dev, nw_out_dev, stats);
    if (stats) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]) == cudaSuccess) stats->sort_ms = ms;
    }
    return s;
}

sph_status sph_autotune(sph_ctx *ctx, const double *h_dev, sph_tuning *best_out)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!h_dev) return fail(ctx, SPH_ERR_INVALID_ARG, "NULL h pointer");
    if (!ctx->sorted) return fail(ctx, SPH_ERR_NOT_SORTED, "sph_sort has not run on this context");
    cudaStream_t st = ctx->stream;
    SegInfo sg = ctx->seg_host;
    sg.nngb = ctx->params.nngb;
    sg.tol = ctx->params.tol;
    *ctx->seg_pinned = sg;
    CU(ctx, cudaMemcpyAsync(ctx->segs, ctx->seg_pinned, sizeof(SegInfo), cudaMemcpyHostToDevice, st),
       "uploading the segment");
    const sph_tuning base = ctx->tuning;
    // one full solve from h_dev with tuning t: its device time in ms (< 0 on failure, with the
    // status in *err)
    auto time_one = [&](const sph_tuning &t, sph_status *err) -> float {
        ctx->tuning = t;
        SolveArgs a = solve_args(ctx);
        *err = SPH_OK;
        cudaError_t e = cudaMemsetAsync(&ctx->ds->status, 0, sizeof(int32_t), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(&ctx->ds->h_varies, 0, sizeof(int32_t), st);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[2], st);
        if (e == cudaSuccess) e = launch_solve_init(a, h_dev, ctx->params.max_iter, st);
        if (e != cudaSuccess) {
            *err = cuda_fail(ctx, e, "autotune solve");
            return -1.f;
        }
        int passes = 0;
        sph_status s = host_passes(ctx, a, false, &passes);
        if (s == SPH_OK) {
            e = cudaEventRecord(ctx->ev[3], st);
            if (e != cudaSuccess) s = cuda_fail(ctx, e, "event");
        }
        if (s == SPH_OK) s = read_state(ctx);
        if (s == SPH_OK && (ctx->ds_host->status | ctx->ds_host->sort_status))
            s = device_status_error(ctx, ctx->ds_host->status | ctx->ds_host->sort_status);
        float ms = -1.f;
        if (s == SPH_OK) {
            e = cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
            if (e != cudaSuccess) s = cuda_fail(ctx, e, "event time");
        }
        *err = s;
        return s == SPH_OK ? ms : -1.f;
    };
    // one knob at a time from the current tuning, two rounds; a change is kept only when it
    // saves more than 1 % (timing noise)
    sph_tuning best = base;
    best.direct_pct = 0;  // FP32 evaluates directly (FP64 always queues)
    sph_status err = SPH_OK;
    float best_ms = time_one(best, &err);
    if (best_ms < 0.f) {
        ctx->tuning = base;
        return err;
    }
    const int mode = ctx->params.precision == SPH_PREC_FP64 ? 0 : 2;
    for (int round = 0; round < 2; round++) {
        for (int knob = 0; knob < 9; knob++) {
            if (knob == 6 && ctx->params.list_entries == 0) continue;  // no lists, no margin
            int vals[4];
            int nv = 0;
            switch (knob) {
            case 0: vals[0] = 0, vals[1] = 16, vals[2] = 32, vals[3] = 64, nv = 4; break;  // item_cap
            case 1: vals[0] = 8, vals[1] = 16, vals[2] = 32, nv = 3; break;                // item_max
            case 2: vals[0] = -1, vals[1] = 0, vals[2] = 1, nv = 3; break;                 // group_shift
            case 3: vals[0] = 2, vals[1] = 3, nv = 2; break;                               // cell_div
            case 4: vals[0] = 128, vals[1] = 256, nv = 2; break;                           // block_threads
            case 6: vals[0] = 5, vals[1] = 10, vals[2] = 20, nv = 3; break;                // list_margin_pct
            case 7: vals[0] = -1, vals[1] = 0, vals[2] = 1, vals[3] = 2, nv = 4; break;    // sparse_shift
            case 8: vals[0] = 0, vals[1] = 1, vals[2] = 4, nv = 3; break;                  // sparse_item_max
            default: {                                                                     // blocks_per_sm
                const int bt = best.block_threads;
                const int ti = bt == 64 ? 0 : bt == 128 ? 1 : 2;
                int &occ = ctx->occupancy[mode][ti];
                if (occ == 0) occ = density_blocks_per_sm(ctx->params.precision, 0, bt);
                vals[0] = 0;
                nv = 1;
                if (occ > 1) vals[nv++] = occ - 1;
            }
            }
            for (int v = 0; v < nv; v++) {
                sph_tuning t = best;
                int *field = knob == 0   ? &t.item_cap
                             : knob == 1 ? &t.item_max
                             : knob == 2 ? &t.group_shift
                             : knob == 3 ? &t.cell_div
                             : knob == 4 ? &t.block_threads
                             : knob == 5 ? &t.blocks_per_sm
                             : knob == 6 ? &t.list_margin_pct
                             : knob == 7 ? &t.sparse_shift
                                         : &t.sparse_item_max;
                if (*field == vals[v]) continue;
                *field = vals[v];
                const float ms = time_one(t, &err);
                if (ms < 0.f) {
                    ctx->tuning = base;
                    return err;
                }
                if (ms < 0.99f * best_ms) {
                    best_ms = ms;
                    best = t;
                }
            }
        }
    }
    ctx->tuning = best;
    cache_store(ctx, ctx->n, best);
    if (best_out) *best_out = best;
    return SPH_OK;
}

sph_status sph_density_eval(sph_ctx *ctx, const double *h_dev, double *rho_out_dev,
                            int32_t *count_out_dev, double *nw_out_dev, double *dnw_out_dev)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!h_dev || !rho_out_dev || !count_out_dev)
        return fail(ctx, SPH_ERR_INVALID_ARG, "NULL h, rho or count pointer");
    if (!ctx->sorted) return fail(ctx, SPH_ERR_NOT_SORTED, "sph_sort has not run on this context");
    cudaStream_t st = ctx->stream;
    SolveArgs a = solve_args(ctx);
    a.lst = nullptr;  // one pass: nothing to reuse
    CU(ctx, cudaMemsetAsync(&ctx->ds->status, 0, sizeof(int32_t), st), "clearing the status word");
    CU(ctx, cudaMemsetAsync(&ctx->ds->h_varies, 0, sizeof(int32_t), st), "clearing the h flag");
    CU(ctx, launch_solve_init(a, h_dev, 1, st), "init");
    sph_status s = read_state(ctx);
    if (s != SPH_OK) return s;
    if (ctx->ds_host->status | ctx->ds_host->sort_status)
        return device_status_error(ctx, ctx->ds_host->status | ctx->ds_host->sort_status);
    CU(ctx, launch_pass(a, 0, false, st), "density pass");
    CU(ctx, launch_scatter(a, nullptr, rho_out_dev, count_out_dev, nw_out_dev, dnw_out_dev, st), "scatter");
    s = read_state(ctx);
    if (s != SPH_OK) return s;
    if (ctx->ds_host->status) return device_status_error(ctx, ctx->ds_host->status);
    return SPH_OK;
}

sph_status sph_neighbours_sampled(sph_ctx *ctx, const double *h_dev, int64_t n_sample,
                                  const int64_t *sample_dev, int32_t max_nbr, int32_t *nbr_dev,
                                  int32_t *nbr_count_dev, double *rho_out_dev, int32_t *count_out_dev)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!h_dev || !sample_dev || !nbr_dev || !nbr_count_dev || !rho_out_dev || !count_out_dev)
        return fail(ctx, SPH_ERR_INVALID_ARG, "NULL pointer argument");
    if (!ctx->sorted) return fail(ctx, SPH_ERR_NOT_SORTED, "sph_sort has not run on this context");
    if (n_sample < 1 || n_sample > ctx->n)
        return fail(ctx, SPH_ERR_INVALID_ARG, "n_sample = %lld outside [1, n = %lld]", (long long)n_sample,
                    (long long)ctx->n);
    if (max_nbr < 1) return fail(ctx, SPH_ERR_INVALID_ARG, "max_nbr must be >= 1");
    if (ctx->params.precision != SPH_PREC_FP64 && ctx->tuning.direct_pct != 0)
        return fail(ctx, SPH_ERR_UNSUPPORTED, "the neighbour export needs direct_pct = 0 in FP32");
    cudaStream_t st = ctx->stream;
    SolveArgs a = solve_args(ctx);
    a.lst = nullptr;  // one pass, searched
    CU(ctx, cudaMemsetAsync(&ctx->ds->status, 0, sizeof(int32_t), st), "clearing the status word");
    CU(ctx, cudaMemsetAsync(&ctx->ds->h_varies, 0, sizeof(int32_t), st), "clearing the h flag");
    CU(ctx, launch_solve_init(a, h_dev, 1, st), "init");
    CU(ctx, launch_nb_setup(a, ctx->nb_slot, sample_dev, n_sample, nbr_count_dev, st), "sample set-up");
    sph_status s = read_state(ctx);
    if (s != SPH_OK) return s;
    {
        const int bits = ctx->ds_host->status | ctx->ds_host->sort_status;
        if (bits & kBadSample) return fail(ctx, SPH_ERR_INVALID_ARG, "a sample index is outside [0, n) or repeated");
        if (bits) return device_status_error(ctx, bits);
    }
    a.nb_slot = ctx->nb_slot;
    a.nb_out = nbr_dev;
    a.nb_cnt = nbr_count_dev;
    a.nb_max = max_nbr;
    CU(ctx, launch_pass(a, 0, false, st), "density pass with the neighbour export");
    CU(ctx, launch_scatter(a, nullptr, rho_out_dev, count_out_dev, nullptr, nullptr, st), "scatter");
    s = read_state(ctx);
    if (s != SPH_OK) return s;
    if (ctx->ds_host->status) return device_status_error(ctx, ctx->ds_host->status);
    return SPH_OK;
}

sph_status sph_interact(sph_ctx *ctx, const double *h_dev, const double *vel_xyz_dev, double *rho_out_dev,
                        double *vmean_xyz_out_dev, double *sigma2_out_dev, double *div_out_dev,
                        double *curl_xyz_out_dev, int32_t *count_out_dev, sph_stats *stats)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!h_dev || !vel_xyz_dev || !rho_out_dev || !vmean_xyz_out_dev || !sigma2_out_dev || !div_out_dev ||
        !curl_xyz_out_dev || !count_out_dev)
        return fail(ctx, SPH_ERR_INVALID_ARG, "NULL pointer argument");
    if (!ctx->sorted) return fail(ctx, SPH_ERR_NOT_SORTED, "sph_sort has not run on this context");
    cudaStream_t st = ctx->stream;
    const int launches0 = ctx->launches;
    SolveArgs a = solve_args(ctx);
    a.lst = nullptr;  // one pass, searched
    CU(ctx, cudaEventRecord(ctx->ev[2], st), "event");
    CU(ctx, cudaMemsetAsync(&ctx->ds->status, 0, sizeof(int32_t), st), "clearing the status word");
    CU(ctx, cudaMemsetAsync(&ctx->ds->h_varies, 0, sizeof(int32_t), st), "clearing the h flag");
    CU(ctx, launch_solve_init(a, h_dev, 1, st), "init");
    CU(ctx, launch_gather_vel(a, vel_xyz_dev, ctx->vrec, st), "velocity records");
    sph_status s = read_state(ctx);
    if (s != SPH_OK) return s;
    if (ctx->ds_host->status | ctx->ds_host->sort_status)
        return device_status_error(ctx, ctx->ds_host->status | ctx->ds_host->sort_status);
    InteractArgs ia{};
    ia.vrec = ctx->vrec;
    ia.vel = vel_xyz_dev;
    ia.rho = rho_out_dev;
    ia.vmean = vmean_xyz_out_dev;
    ia.sigma2 = sigma2_out_dev;
    ia.div = div_out_dev;
    ia.curl = curl_xyz_out_dev;
    ia.count = count_out_dev;
    a.dens_ev[0] = ctx->dev_ev[0];
    a.dens_ev[1] = ctx->dev_ev[1];
    CU(ctx, launch_interact_pass(a, ia, st), "interaction pass");
    CU(ctx, cudaEventRecord(ctx->ev[3], st), "event");
    s = read_state(ctx);
    if (s != SPH_OK) return s;
    if (ctx->ds_host->status) return device_status_error(ctx, ctx->ds_host->status);
    if (stats) {
        const DevState &d = *ctx->ds_host;
        *stats = sph_stats{};
        stats->passes = 1;
        stats->kernel_launches = ctx->launches - launches0;
        stats->todo_per_pass[0] = ctx->n;
        stats->pair_evals = (int64_t)d.pair_evals;
        stats->pair_tests = (int64_t)d.pair_tests;
        stats->pairs_per_pass[0] = (int64_t)d.pair_evals;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
        stats->solve_ms = ms;
        if (cudaEventElapsedTime(&ms, ctx->dev_ev[0], ctx->dev_ev[1]) == cudaSuccess) {
            stats->density_ms = ms;
            stats->density_ms_per_pass[0] = ms;
        }
        stats->density_launches = 1;
    }
    return SPH_OK;
}

sph_status sph_knn_solve(sph_ctx *ctx, int32_t k, double *h_inout_dev, double *rho_out_dev,
                         int32_t *count_out_dev, double *nw_out_dev, sph_stats *stats)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    if (!h_inout_dev || !rho_out_dev || !count_out_dev)
        return fail(ctx, SPH_ERR_INVALID_ARG, "NULL h, rho or count pointer");
    if (!ctx->sorted) return fail(ctx, SPH_ERR_NOT_SORTED, "sph_sort has not run on this context");
    if (ctx->kl.seg_bits > 0)
        return fail(ctx, SPH_ERR_UNSUPPORTED, "sph_knn_solve runs on the particles of sph_sort, not on "
                                              "batched groups");
    if (k < 2 || k > SPH_KNN_MAX_K || (int64_t)k > ctx->n)
        return fail(ctx, SPH_ERR_INVALID_ARG, "k = %d outside [2, min(%d, n = %lld)]", k, SPH_KNN_MAX_K,
                    (long long)ctx->n);
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t st = ctx->stream;
    const int launches0 = ctx->launches;
    SolveArgs a = solve_args(ctx);
    a.free_first = 0;  // the density pass of leftover particles keeps the body under its test
    a.lst = nullptr;
    CU(ctx, cudaEventRecord(ctx->ev[2], st), "event");
    CU(ctx, cudaMemsetAsync(&ctx->ds->status, 0, sizeof(int32_t), st), "clearing the status word");
    CU(ctx, launch_knn_init(a, h_inout_dev, ctx->params.max_iter, k, st), "init");
    sph_status s = read_state(ctx);
    if (s != SPH_OK) return s;
    if (ctx->ds_host->status | ctx->ds_host->sort_status)
        return device_status_error(ctx, ctx->ds_host->status | ctx->ds_host->sort_status);
    // selection passes over the shrinking todo list
    int cur = 0, passes_run = 0;
    for (int pass = 0; pass < ctx->params.max_iter; pass++) {
        a.dens_ev[0] = ctx->dev_ev[2 * pass];
        a.dens_ev[1] = ctx->dev_ev[2 * pass + 1];
        CU(ctx, launch_knn_pass(a, cur, k, st), "kNN pass");
        passes_run = pass + 1;
        CU(ctx, cudaMemcpyAsync(&ctx->ds_host->todo_count, &ctx->ds->todo_count, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st),
           "reading the todo count");
        CU(ctx, cudaStreamSynchronize(st), "synchronising the pass");
        cur = 1 - cur;
        if (ctx->ds_host->todo_count == 0) break;
    }
    s = read_state(ctx);
    if (s != SPH_OK) return s;
    const DevState knn = *ctx->ds_host;
    if (knn.status) return device_status_error(ctx, knn.status);
    // the density of particles without a selection, at their last radius
    a.dens_ev[0] = a.dens_ev[1] = nullptr;
    CU(ctx, launch_knn_finish(a, st), "kNN finish");
    CU(ctx, launch_scatter(a, h_inout_dev, rho_out_dev, count_out_dev, nw_out_dev, nullptr, st), "scatter");
    CU(ctx, cudaEventRecord(ctx->ev[3], st), "event");
    s = read_state(ctx);
    if (s != SPH_OK) return s;
    const DevState &d = *ctx->ds_host;
    if (d.status) return device_status_error(ctx, d.status);
    if (stats) {
        stats->passes = knn.pass;
        stats->kernel_launches = ctx->launches - launches0 + ctx->sort_launches;
        for (int q = 0; q < SPH_MAX_PASSES; q++)
            stats->todo_per_pass[q] = q < knn.pass ? knn.todo_per_pass[q] : 0;
        stats->unconverged = knn.todo_count;
        stats->exceeded = knn.exceeded;
        stats->pair_evals = (int64_t)knn.pair_evals;
        stats->pair_tests = (int64_t)knn.pair_tests;
        for (int q = 0; q < SPH_MAX_PASSES; q++)
            stats->pairs_per_pass[q] = q < knn.pass ? (int64_t)knn.pairs_per_pass[q] : 0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]);
        stats->solve_ms = ms;
        if (cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]) == cudaSuccess) stats->sort_ms = ms;
        double kms = 0.0;
        for (int q = 0; q < passes_run; q++) {
            float m = 0.f;
            if (cudaEventElapsedTime(&m, ctx->dev_ev[2 * q], ctx->dev_ev[2 * q + 1]) == cudaSuccess) {
                kms += m;
                stats->density_ms_per_pass[q] = m;
            }
        }
        stats->density_ms = kms;
        stats->density_launches = passes_run;
    }
    if (knn.exceeded > 0)
        return fail(ctx, SPH_ERR_H_EXCEEDS_BOX, "%d particles: the K-th neighbour lies at or beyond min(box)/2",
                    knn.exceeded);
    if (knn.todo_count > 0)
        return fail(ctx, SPH_ERR_NOT_CONVERGED, "%d particles without a selection after %d passes",
                    knn.todo_count, knn.pass);
    return SPH_OK;
}

sph_status sph_batch_solve(sph_ctx *ctx, int64_t n_groups, const int64_t *offsets_dev,
                           const double *pos_xyz_dev, const double *mass_dev, const double *nngb_dev,
                           const double *tol_dev, double *h_inout_dev, double *rho_out_dev,
                           int32_t *count_out_dev, double *nw_out_dev, sph_stats *stats)
{
    if (!ctx) return SPH_ERR_INVALID_ARG;
    ctx->sorted = false;
    if (!offsets_dev || !pos_xyz_dev || !mass_dev || !nngb_dev || !tol_dev || !h_inout_dev ||
        !rho_out_dev || !count_out_dev)
        return fail(ctx, SPH_ERR_INVALID_ARG, "NULL pointer argument");
    if (n_groups < 1) return fail(ctx, SPH_ERR_INVALID_ARG, "n_groups must be >= 1");
    if (n_groups > ctx->max_groups)
        return fail(ctx, SPH_ERR_OOM, "n_groups = %lld exceeds the context limit %lld",
                    (long long)n_groups, (long long)ctx->max_groups);
    if (stats) memset(stats, 0, sizeof(*stats));
    cudaStream_t st = ctx->stream;
    CU(ctx, cudaMemcpyAsync(ctx->i64_pinned, offsets_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, st),
       "reading offsets[0]");
    CU(ctx, cudaMemcpyAsync(ctx->i64_pinned + 1, offsets_dev + n_groups, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, st),
       "reading offsets[n_groups]");
    CU(ctx, cudaStreamSynchronize(st), "synchronising");
    const int64_t n = ctx->i64_pinned[1];
    if (ctx->i64_pinned[0] != 0) return fail(ctx, SPH_ERR_INVALID_ARG, "offsets[0] must be 0");
    if (n < 1) return fail(ctx, SPH_ERR_INVALID_ARG, "offsets[n_groups] must be >= 1");
    if (n > ctx->capacity)
        return fail(ctx, SPH_ERR_OOM, "n = %lld exceeds the context capacity %lld", (long long)n,
                    (long long)ctx->capacity);
    ctx->n = n;
    int seg_bits = 0;
    while ((1ll << seg_bits) < n_groups) seg_bits++;
    ctx->kl.seg_bits = seg_bits;
    ctx->kl.lmax = std::min(21, (63 - seg_bits) / 3);
    ctx->kl.key_bits = seg_bits + 3 * ctx->kl.lmax;
    ctx->kl.coord_bits = 31;

    CU(ctx, cudaEventRecord(ctx->ev[0], st), "event");
    CU(ctx, cudaMemsetAsync(ctx->ds, 0, sizeof(DevState), st), "clearing the device state");
    const int launches0 = ctx->launches;
    SortArgs a = sort_args(ctx);
    CU(ctx, launch_group_setup(a, n_groups, offsets_dev, pos_xyz_dev, n, nngb_dev, tol_dev, ctx->tsize,
                               ctx->toff, st),
       "group setup");
    const bool fp64 = ctx->params.precision == SPH_PREC_FP64;
    uint4 *rec = fp64 ? nullptr : (uint4 *)ctx->pdbl;
    CU(ctx, launch_keys_open(a, n, pos_xyz_dev, mass_dev, offsets_dev, n_groups, st, rec), "morton keys");
    int which = 0;
    CU(ctx, launch_radix_sort(a, n, &which, st), "radix sort");
    ctx->which = which;
    if (fp64)
        CU(ctx, launch_gather_open(a, n, pos_xyz_dev, mass_dev, ctx->idx[which], ctx->key[which], st), "gather");
    else
        CU(ctx, launch_gather_rec(a, n, ctx->idx[which], rec, st), "gather");
    ctx->fp64_records = fp64;
    CU(ctx, launch_cell_table(a, n, ctx->key[which], st), "cell table");
    CU(ctx, cudaEventRecord(ctx->ev[1], st), "event");
    ctx->sort_launches = ctx->launches - launches0;
    sph_status s = SPH_OK;
    if (!ctx->params.use_graph) {
        s = read_state(ctx);
        if (s != SPH_OK) return s;
        if (ctx->ds_host->sort_status) return device_status_error(ctx, ctx->ds_host->sort_status);
    }
    s = run_solve(ctx, h_inout_dev, rho_out_dev, count_out_dev, nw_out_dev, stats);
    if (stats) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]) == cudaSuccess) stats->sort_ms = ms;
    }
    return s;
}

}  // extern "C"
