// sph_static_eval.cu -- sph_density_eval_static: the fixed-h density evaluation (spatial
// sort + one density pass) for callers that cannot allocate device memory.
//
// Why it exists.  Some programs that would call this library must not call cudaMalloc or
// cudaFree on that code path: a plugin running inside a host application that owns all
// device memory through its own pool (a raw cudaMalloc would fail or fragment that pool),
// or a latency-critical loop where cudaFree would stall every stream on the device.  The
// context API allocates its scratch once in sph_create; this entry point instead uses one
// fixed array of device memory that is part of the library image itself.
//
// What it costs.  The array below is reserved on every GPU that loads the library and
// stays there until the process exits (about 5 MB).  Its size caps the particle count at
// SPH_STATIC_MAX_PARTICLES.  All calls share the one array: two calls whose work overlaps
// on the GPU (different streams, different host threads) corrupt each other's results,
// so callers must serialise them.  The array keeps the previous call's contents; the only
// part that must start at zero (the device state word) is cleared by every call.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>

#include "sph.h"
#include "sph_kernels.cuh"

using namespace sph;

namespace {

constexpr int64_t kMaxN = SPH_STATIC_MAX_PARTICLES;
constexpr size_t kAlign = 256;

constexpr size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Upper bounds of the buffer sizes for kMaxN particles (checked against the launchers'
// own size functions at set-up).
constexpr int64_t kHistEntries = 256 * ((kMaxN + 2047) / 2048 + 1);
constexpr int64_t kAuxEntries = ((kHistEntries > kMaxN ? kHistEntries : kMaxN) + 2047) / 2048 + 2 + 8;
constexpr int64_t kTabEntries = kMaxN + 2;

constexpr size_t kScratchBytes =
    2 * up(kMaxN * 8) + 2 * up(kMaxN * 4)          // keys, indices (ping-pong)
    + 2 * up(kHistEntries * 4) + up(kAuxEntries * 4)  // radix histograms, scan scratch
    + up(kMaxN * 16) + up(kMaxN * 32)                // sorted fixed-point and FP64 records
    + up(kTabEntries * 4) + up(sizeof(SegInfo))      // cell table, segment descriptor
    + 7 * up(kMaxN * 8) + up(kMaxN * 4)              // h state and evaluation outputs
    + 4 * up(kMaxN * 4)                              // FP32 copies of h and of the outputs
    + 2 * up(kMaxN * 4) + up(kMaxN * 4) + up((kMaxN + 1) * 4)  // todo lists, flags, items
    + up(sizeof(DevState));

// The scratch itself: device memory that is part of the loaded library image.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool done = false;
    unsigned char *base = nullptr;  // device address of g_static_scratch on this device
    int num_sms = 0;
    int density_grid[2] = {0, 0};
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

struct Carved {
    uint64_t *key[2];
    int32_t *idx[2];
    int32_t *hist, *hist_off, *aux;
    uint4 *pfix;
    double4_32a *pdbl;
    int32_t *ctab;
    SegInfo *segs;
    double *h, *hlo, *hhi, *e_h, *e_rho, *e_nw, *e_dnw;
    int32_t *e_cnt, *todo[2], *flags, *items;
    float *h32, *e_rho32, *e_nw32, *e_dnw32;
    DevState *ds;
};

Carved carve(unsigned char *base)
{
    Carved c{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *p = base + off;
        off += up(bytes);
        return p;
    };
    for (int k = 0; k < 2; k++) c.key[k] = (uint64_t *)take(kMaxN * 8);
    for (int k = 0; k < 2; k++) c.idx[k] = (int32_t *)take(kMaxN * 4);
    c.hist = (int32_t *)take(kHistEntries * 4);
    c.hist_off = (int32_t *)take(kHistEntries * 4);
    c.aux = (int32_t *)take(kAuxEntries * 4);
    c.pfix = (uint4 *)take(kMaxN * 16);
    c.pdbl = (double4_32a *)take(kMaxN * 32);
    c.ctab = (int32_t *)take(kTabEntries * 4);
    c.segs = (SegInfo *)take(sizeof(SegInfo));
    c.h = (double *)take(kMaxN * 8);
    c.hlo = (double *)take(kMaxN * 8);
    c.hhi = (double *)take(kMaxN * 8);
    c.e_h = (double *)take(kMaxN * 8);
    c.e_rho = (double *)take(kMaxN * 8);
    c.e_nw = (double *)take(kMaxN * 8);
    c.e_dnw = (double *)take(kMaxN * 8);
    c.e_cnt = (int32_t *)take(kMaxN * 4);
    c.h32 = (float *)take(kMaxN * 4);
    c.e_rho32 = (float *)take(kMaxN * 4);
    c.e_nw32 = (float *)take(kMaxN * 4);
    c.e_dnw32 = (float *)take(kMaxN * 4);
    for (int k = 0; k < 2; k++) c.todo[k] = (int32_t *)take(kMaxN * 4);
    c.flags = (int32_t *)take(kMaxN * 4);
    c.items = (int32_t *)take((kMaxN + 1) * 4);
    c.ds = (DevState *)take(sizeof(DevState));
    return c;
}

// Once per device, with that device current: look up the device address of the array
// (host code cannot use the symbol's name as a pointer) and the persistent grid sizes.
sph_status setup_current_device(DeviceSetup **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPH_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SPH_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return SPH_ERR_CUDA;
        }
        if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SPH_ERR_CUDA;
        // the launchers' own size rules must fit the reserved regions
        if (radix_hist_size(kMaxN) > kHistEntries ||
            scan_aux_size(kHistEntries > kMaxN ? kHistEntries : kMaxN) + 8 > kAuxEntries)
            return SPH_ERR_UNSUPPORTED;
        s.base = (unsigned char *)ptr;
        s.density_grid[0] = s.num_sms * density_blocks_per_sm(SPH_PREC_FP64, 0);
        s.density_grid[1] = s.num_sms * density_blocks_per_sm(SPH_PREC_FP32_KAHAN, 0);
        s.done = true;
    }
    *out = &s;
    return SPH_OK;
}

#define CUS(expr)                                                                            \
    do {                                                                                     \
        if ((expr) != cudaSuccess) return SPH_ERR_CUDA;                                      \
    } while (0)

}  // namespace

extern "C" sph_status sph_density_eval_static(const sph_params *params, int64_t n,
                                               const double *pos_xyz_dev, const double *mass_dev,
                                               const double *h_dev, void *cuda_stream,
                                               double *rho_out_dev, int32_t *count_out_dev,
                                               double *nw_out_dev, double *dnw_out_dev)
{
    if (!params || !pos_xyz_dev || !mass_dev || !h_dev || !rho_out_dev || !count_out_dev)
        return SPH_ERR_INVALID_ARG;
    if (n < 1) return SPH_ERR_INVALID_ARG;
    if (n > kMaxN) return SPH_ERR_OOM;  // beyond the fixed array: no fallback allocation
    if (params->kernel != SPH_KERNEL_M4) return SPH_ERR_UNSUPPORTED;
    if (params->periodic != 1) return SPH_ERR_UNSUPPORTED;
    if (params->precision != SPH_PREC_FP64 && params->precision != SPH_PREC_FP32_KAHAN)
        return SPH_ERR_INVALID_ARG;
    for (int d = 0; d < 3; d++)
        if (!(params->box[d] > 0.0 && params->box[d] <= DBL_MAX)) return SPH_ERR_INVALID_ARG;

    DeviceSetup *dev = nullptr;
    sph_status s = setup_current_device(&dev);
    if (s != SPH_OK) return s;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Carved c = carve(dev->base);
    int launches = 0;

    KeyLayout kl{};
    kl.lmax = 21;
    kl.seg_bits = 0;
    kl.key_bits = 63;
    kl.coord_bits = 32;
    SegInfo sg;
    memset(&sg, 0, sizeof(sg));
    for (int d = 0; d < 3; d++) {
        sg.q[d] = std::ldexp(params->box[d], -32);
        sg.inv_q[d] = std::ldexp(1.0 / params->box[d], 32);
        sg.box[d] = params->box[d];
    }
    sg.nngb = params->nngb;
    sg.tol = params->tol;
    sg.half_box = 0.5 * fmin(params->box[0], fmin(params->box[1], params->box[2]));
    sg.periodic = 1;
    int lc = 0;
    while (lc < 10 && (1ll << (3 * (lc + 1))) <= n) lc++;
    sg.level_c = lc;
    sg.start = 0;
    sg.end = (int32_t)n;

    // the segment descriptor comes from pageable host memory (staged by the CUDA driver, no
    // allocation here); the state word must start at zero
    CUS(cudaMemcpyAsync(c.segs, &sg, sizeof(SegInfo), cudaMemcpyHostToDevice, st));
    CUS(cudaMemsetAsync(c.ds, 0, sizeof(DevState), st));

    SortArgs sa{};
    for (int k = 0; k < 2; k++) {
        sa.key[k] = c.key[k];
        sa.idx[k] = c.idx[k];
    }
    sa.hist = c.hist;
    sa.hist_off = c.hist_off;
    sa.scan_aux = c.aux;
    sa.pfix = c.pfix;
    sa.pdbl = c.pdbl;
    sa.ctab = c.ctab;
    sa.segs = c.segs;
    sa.ds = c.ds;
    sa.kl = kl;
    sa.grid_cap = dev->num_sms * 16;
    sa.table_extra = 0;
    sa.self_floor = 32.0 / 3.0;
    sa.launches = &launches;
    CUS(launch_keys_periodic(sa, n, pos_xyz_dev, mass_dev, sg, params->box, st));
    int which = 0;
    CUS(launch_radix_sort(sa, n, &which, st));
    CUS(launch_gather_periodic(sa, n, pos_xyz_dev, mass_dev, c.idx[which], sg, st));
    CUS(launch_cell_table(sa, n, c.key[which], st));

    SolveArgs a{};
    a.pfix = c.pfix;
    a.pdbl = c.pdbl;
    a.key = c.key[which];
    a.idx = c.idx[which];
    a.segs = c.segs;
    a.ctab = c.ctab;
    a.kl = kl;
    a.n = n;
    a.h = c.h;
    a.hlo = c.hlo;
    a.hhi = c.hhi;
    a.e_h = c.e_h;
    a.e_rho = c.e_rho;
    a.e_nw = c.e_nw;
    a.e_dnw = c.e_dnw;
    a.e_cnt = c.e_cnt;
    a.h32 = c.h32;
    a.e_rho32 = c.e_rho32;
    a.e_nw32 = c.e_nw32;
    a.e_dnw32 = c.e_dnw32;
    a.todo[0] = c.todo[0];
    a.todo[1] = c.todo[1];
    a.flags = c.flags;
    a.items = c.items;
    a.scan_aux = c.aux;
    a.ds = c.ds;
    a.grid_cap = dev->num_sms * 16;
    a.precision = params->precision;
    a.kernel = SPH_KERNEL_M4;
    a.density_grid = dev->density_grid[params->precision == SPH_PREC_FP64 ? 0 : 1];
    a.gmax = 32;
    a.gmax_sparse = 32;
    a.group_shift = 1;
    a.cell_div = 3;
    a.direct_pct = 0;
    a.launches = &launches;
    CUS(launch_solve_init(a, h_dev, 1, st));

    // The sort flags bad positions and masses, the init flags a bad h.  Read the state word
    // (into pageable host memory) and stop before the density pass if either is set: the
    // pass's cell enumeration relies on every h lying in (0, min(box)/2).
    DevState host{};
    CUS(cudaMemcpyAsync(&host, c.ds, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CUS(cudaStreamSynchronize(st));
    if (host.status | host.sort_status) return SPH_ERR_DEVICE_STATUS;

    CUS(launch_pass(a, 0, false, st));
    CUS(launch_scatter(a, nullptr, rho_out_dev, count_out_dev, nw_out_dev, dnw_out_dev, st));

    // wait for the results and read the state word again
    CUS(cudaMemcpyAsync(&host, c.ds, sizeof(DevState), cudaMemcpyDeviceToHost, st));
    CUS(cudaStreamSynchronize(st));
    if (host.status | host.sort_status) return SPH_ERR_DEVICE_STATUS;
    return SPH_OK;
}
