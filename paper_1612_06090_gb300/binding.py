"""ctypes binding of libsph.so (include/sph.h).

Argument marshalling only: every step of the solve runs in the CUDA library.  The raw
functions keep the C names and take device pointers as Python ints (``tensor.data_ptr()``)
and a CUDA stream handle (``torch.cuda.current_stream().cuda_stream``).  ``Solver`` wraps a
context for torch tensors.  If libsph.so is missing the binding raises; nothing falls back
to the CPU.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsph.so")

# sph_status
SPH_OK = 0
SPH_ERR_INVALID_ARG = 1
SPH_ERR_CUDA = 2
SPH_ERR_OOM = 3
SPH_ERR_NOT_SORTED = 4
SPH_ERR_H_EXCEEDS_BOX = 5
SPH_ERR_NOT_CONVERGED = 6
SPH_ERR_DEVICE_STATUS = 7
SPH_ERR_UNSUPPORTED = 8
# sph_kernel / sph_precision
SPH_KERNEL_M4 = 0
SPH_KERNEL_WENDLAND_C6 = 1
SPH_PREC_FP64 = 0
SPH_PREC_FP32_KAHAN = 1
SPH_MAX_PASSES = 64

EXPORTED = ("sph_create", "sph_set_params", "sph_sort", "sph_density_solve", "sph_density_eval",
            "sph_knn_solve",
            "sph_batch_solve", "sph_destroy", "sph_status_string", "sph_last_error",
            "sph_density_eval_static", "sph_get_tuning", "sph_set_tuning", "sph_autotune",
            "sph_neighbours_sampled", "sph_interact")
SPH_STATIC_MAX_PARTICLES = 32768
SPH_KNN_MAX_K = 512


class SphParams(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("periodic", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("nngb", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("list_entries", ctypes.c_int32),
        ("tune_cache", ctypes.c_char_p),
    ]


class SphStats(ctypes.Structure):
    _fields_ = [
        ("passes", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int32),
        ("todo_per_pass", ctypes.c_int64 * SPH_MAX_PASSES),
        ("unconverged", ctypes.c_int64),
        ("exceeded", ctypes.c_int64),
        ("pair_evals", ctypes.c_int64),
        ("sort_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("density_ms", ctypes.c_double),
        ("density_launches", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("pair_tests", ctypes.c_int64),
        ("pairs_per_pass", ctypes.c_int64 * SPH_MAX_PASSES),
        ("density_ms_per_pass", ctypes.c_double * SPH_MAX_PASSES),
        ("list_evals", ctypes.c_int64),
    ]

    def to_dict(self) -> dict:
        p = int(self.passes)
        return {
            "passes": p,
            "kernel_launches": int(self.kernel_launches),
            "todo_per_pass": [int(v) for v in self.todo_per_pass[: max(0, min(p, SPH_MAX_PASSES))]],
            "unconverged": int(self.unconverged),
            "exceeded": int(self.exceeded),
            "pair_evals": int(self.pair_evals),
            "sort_ms": float(self.sort_ms),
            "solve_ms": float(self.solve_ms),
            "density_ms": float(self.density_ms),
            "density_launches": int(self.density_launches),
            "pair_tests": int(self.pair_tests),
            "pairs_per_pass": [int(v) for v in self.pairs_per_pass[: max(0, min(p, SPH_MAX_PASSES))]],
            "density_ms_per_pass": [float(v) for v in self.density_ms_per_pass[: max(0, min(p, SPH_MAX_PASSES))]],
            "list_evals": int(self.list_evals),
        }


class SphTuning(ctypes.Structure):
    _fields_ = [
        ("group_shift", ctypes.c_int32),
        ("cell_div", ctypes.c_int32),
        ("table_extra", ctypes.c_int32),
        ("direct_pct", ctypes.c_int32),
        ("item_cap", ctypes.c_int32),
        ("item_max", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("list_margin_pct", ctypes.c_int32),
        ("sparse_shift", ctypes.c_int32),
        ("sparse_item_max", ctypes.c_int32),
    ]

    def to_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load libsph.so (built by paper_1612_06090_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1612_06090_gb300.build` (nvcc, sm_103a)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.sph_create.restype = i32
    L.sph_create.argtypes = [ctypes.POINTER(SphParams), i64, vp, ctypes.POINTER(vp)]
    L.sph_set_params.restype = i32
    L.sph_set_params.argtypes = [vp, ctypes.POINTER(SphParams)]
    L.sph_sort.restype = i32
    L.sph_sort.argtypes = [vp, i64, vp, vp]
    L.sph_density_solve.restype = i32
    L.sph_density_solve.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(SphStats)]
    L.sph_knn_solve.restype = i32
    L.sph_knn_solve.argtypes = [vp, i32, vp, vp, vp, vp, ctypes.POINTER(SphStats)]
    L.sph_density_eval.restype = i32
    L.sph_density_eval.argtypes = [vp, vp, vp, vp, vp, vp]
    L.sph_batch_solve.restype = i32
    L.sph_batch_solve.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(SphStats)]
    L.sph_destroy.restype = None
    L.sph_destroy.argtypes = [vp]
    L.sph_status_string.restype = ctypes.c_char_p
    L.sph_status_string.argtypes = [i32]
    L.sph_last_error.restype = ctypes.c_char_p
    L.sph_last_error.argtypes = [vp]
    L.sph_get_tuning.restype = i32
    L.sph_get_tuning.argtypes = [vp, ctypes.POINTER(SphTuning)]
    L.sph_set_tuning.restype = i32
    L.sph_set_tuning.argtypes = [vp, ctypes.POINTER(SphTuning)]
    L.sph_autotune.restype = i32
    L.sph_autotune.argtypes = [vp, vp, ctypes.POINTER(SphTuning)]
    L.sph_neighbours_sampled.restype = i32
    L.sph_neighbours_sampled.argtypes = [vp, vp, i64, vp, i32, vp, vp, vp, vp]
    L.sph_interact.restype = i32
    L.sph_interact.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(SphStats)]
    L.sph_density_eval_static.restype = i32
    L.sph_density_eval_static.argtypes = [ctypes.POINTER(SphParams), i64, vp, vp, vp, vp, vp, vp, vp, vp]
    _lib = L
    return L


def make_params(box=(1.0, 1.0, 1.0), periodic=True, nngb=64.0, tol=2.0, max_iter=64,
                precision=SPH_PREC_FP32_KAHAN, use_graph=False, kernel=SPH_KERNEL_M4,
                tune_cache=None, list_entries=0) -> SphParams:
    p = SphParams()
    for d in range(3):
        p.box[d] = float(box[d])
    p.periodic = int(bool(periodic))
    p.kernel = int(kernel)
    p.nngb = float(nngb)
    p.tol = float(tol)
    p.max_iter = int(max_iter)
    p.precision = int(precision)
    p.use_graph = int(bool(use_graph))
    p.list_entries = int(list_entries)
    p.tune_cache = tune_cache.encode() if tune_cache else None
    return p


# ---- raw C calls (same names as the ABI) -------------------------------------------------

def sph_create(params: SphParams, capacity: int, stream: int = 0):
    out = ctypes.c_void_p()
    st = lib().sph_create(ctypes.byref(params), int(capacity), ctypes.c_void_p(stream or None),
                          ctypes.byref(out))
    return st, out.value


def sph_get_tuning(ctx):
    t = SphTuning()
    st = lib().sph_get_tuning(ctypes.c_void_p(ctx), ctypes.byref(t))
    return st, t


def sph_set_tuning(ctx, tuning: SphTuning) -> int:
    return lib().sph_set_tuning(ctypes.c_void_p(ctx), ctypes.byref(tuning))


def sph_autotune(ctx, h_ptr: int):
    t = SphTuning()
    st = lib().sph_autotune(ctypes.c_void_p(ctx), ctypes.c_void_p(h_ptr or None), ctypes.byref(t))
    return st, t


def sph_set_params(ctx, params: SphParams) -> int:
    return lib().sph_set_params(ctypes.c_void_p(ctx), ctypes.byref(params))


def sph_sort(ctx, n: int, pos_xyz_ptr: int, mass_ptr: int) -> int:
    return lib().sph_sort(ctypes.c_void_p(ctx), int(n), ctypes.c_void_p(pos_xyz_ptr or None),
                          ctypes.c_void_p(mass_ptr or None))


def sph_density_solve(ctx, h_ptr: int, rho_ptr: int, count_ptr: int, nw_ptr: int = 0, stats=None) -> int:
    return lib().sph_density_solve(ctypes.c_void_p(ctx), ctypes.c_void_p(h_ptr or None),
                                   ctypes.c_void_p(rho_ptr or None), ctypes.c_void_p(count_ptr or None),
                                   ctypes.c_void_p(nw_ptr or None),
                                   ctypes.byref(stats) if stats is not None else None)


def sph_knn_solve(ctx, k: int, h_ptr: int, rho_ptr: int, count_ptr: int, nw_ptr: int = 0, stats=None) -> int:
    return lib().sph_knn_solve(ctypes.c_void_p(ctx), int(k), ctypes.c_void_p(h_ptr or None),
                               ctypes.c_void_p(rho_ptr or None), ctypes.c_void_p(count_ptr or None),
                               ctypes.c_void_p(nw_ptr or None),
                               ctypes.byref(stats) if stats is not None else None)


def sph_density_eval(ctx, h_ptr: int, rho_ptr: int, count_ptr: int, nw_ptr: int = 0, dnw_ptr: int = 0) -> int:
    return lib().sph_density_eval(ctypes.c_void_p(ctx), ctypes.c_void_p(h_ptr or None),
                                  ctypes.c_void_p(rho_ptr or None), ctypes.c_void_p(count_ptr or None),
                                  ctypes.c_void_p(nw_ptr or None), ctypes.c_void_p(dnw_ptr or None))


def sph_neighbours_sampled(ctx, h_ptr: int, n_sample: int, sample_ptr: int, max_nbr: int, nbr_ptr: int,
                           nbr_count_ptr: int, rho_ptr: int, count_ptr: int) -> int:
    v = lambda p: ctypes.c_void_p(p or None)  # noqa: E731
    return lib().sph_neighbours_sampled(ctypes.c_void_p(ctx), v(h_ptr), int(n_sample), v(sample_ptr),
                                        int(max_nbr), v(nbr_ptr), v(nbr_count_ptr), v(rho_ptr),
                                        v(count_ptr))


def sph_interact(ctx, h_ptr: int, vel_xyz_ptr: int, rho_ptr: int, vmean_xyz_ptr: int, sigma2_ptr: int,
                 div_ptr: int, curl_xyz_ptr: int, count_ptr: int, stats=None) -> int:
    v = lambda p: ctypes.c_void_p(p or None)  # noqa: E731
    return lib().sph_interact(ctypes.c_void_p(ctx), v(h_ptr), v(vel_xyz_ptr), v(rho_ptr), v(vmean_xyz_ptr),
                              v(sigma2_ptr), v(div_ptr), v(curl_xyz_ptr), v(count_ptr),
                              ctypes.byref(stats) if stats is not None else None)


def sph_batch_solve(ctx, n_groups: int, offsets_ptr: int, pos_xyz_ptr: int, mass_ptr: int,
                    nngb_ptr: int, tol_ptr: int, h_ptr: int, rho_ptr: int, count_ptr: int,
                    nw_ptr: int = 0, stats=None) -> int:
    v = lambda p: ctypes.c_void_p(p or None)  # noqa: E731
    return lib().sph_batch_solve(ctypes.c_void_p(ctx), int(n_groups), v(offsets_ptr), v(pos_xyz_ptr),
                                 v(mass_ptr), v(nngb_ptr), v(tol_ptr), v(h_ptr), v(rho_ptr),
                                 v(count_ptr), v(nw_ptr),
                                 ctypes.byref(stats) if stats is not None else None)


def sph_destroy(ctx) -> None:
    if ctx:
        lib().sph_destroy(ctypes.c_void_p(ctx))


def sph_status_string(status: int) -> str:
    return lib().sph_status_string(int(status)).decode()


def sph_last_error(ctx) -> str:
    r = lib().sph_last_error(ctypes.c_void_p(ctx) if ctx else None)
    return r.decode() if r else ""


def sph_density_eval_static(params: SphParams, n: int, pos_xyz_ptr: int, mass_ptr: int, h_ptr: int,
                            stream: int, rho_ptr: int, count_ptr: int, nw_ptr: int = 0,
                            dnw_ptr: int = 0) -> int:
    """Sort + fixed-h evaluation with no device allocation (scratch is a fixed array in the
    library image, up to SPH_STATIC_MAX_PARTICLES particles; calls must not overlap)."""
    v = lambda p: ctypes.c_void_p(p or None)  # noqa: E731
    return lib().sph_density_eval_static(ctypes.byref(params), int(n), v(pos_xyz_ptr), v(mass_ptr),
                                         v(h_ptr), v(stream), v(rho_ptr), v(count_ptr), v(nw_ptr),
                                         v(dnw_ptr))


# ---- convenience wrapper for torch tensors ------------------------------------------------

class SphError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{sph_status_string(status)} ({status}): {message}")
        self.status = status


def check_tensor(t, name: str, dtype, shape=None, device=None, ndim=None, cuda=True):
    """Reject a tensor the library would misread: it receives bare device pointers and reads
    or writes exactly the documented number of elements of the documented type, so a wrong
    dtype, size or device would be read past its end, overrun or dereferenced on the wrong GPU.
    Checked in this order: a tensor, dtype, number of dimensions, shape, then (cuda=True) the
    CUDA device.  Raises TypeError (not a tensor, wrong dtype) or ValueError (the rest)."""
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dimension(s), got shape {tuple(t.shape)}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if cuda and (t.device.type != "cuda" or (device is not None and t.device.index != device)):
        raise ValueError(f"{name} must be on the context's CUDA device cuda:{device}, got {t.device}")


class Solver:
    """One context on the current CUDA device and stream, driven with torch tensors.

    Positions are a (3, N) float64 CUDA tensor (x, y, z planes), masses (N,) float64.
    solve()/batch_solve() return a dict with h, rho, count, nw, status and stats; a solve
    that ends NOT_CONVERGED or H_EXCEEDS_BOX still returns (check ``status``); any other
    failure raises SphError.
    """

    def __init__(self, capacity: int, stream=None, **params):
        import torch

        self._torch = torch
        self.params = make_params(**params)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        st, ctx = sph_create(self.params, capacity, s.cuda_stream)
        if st != SPH_OK:
            raise SphError(st, "sph_create failed")
        self.ctx = ctx
        self.device = torch.cuda.current_device()
        self.n = 0  # particles of the last successful sph_sort (0: none)

    def close(self):
        if getattr(self, "ctx", None):
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, ok=(SPH_OK,)):
        if st not in ok:
            raise SphError(st, sph_last_error(self.ctx))
        return st

    def _per_particle(self, t, name, dtype=None, cuda=True):
        """A per-particle array of the sorted set.  Before any sort the length is not checked:
        the library then answers NOT_SORTED without touching the arrays."""
        dtype = dtype if dtype is not None else self._torch.float64
        check_tensor(t, name, dtype, (self.n,) if self.n > 0 else None, self.device, ndim=1, cuda=cuda)

    def tuning(self) -> dict:
        st, t = sph_get_tuning(self.ctx)
        self._check(st)
        return t.to_dict()

    def set_tuning(self, **kw):
        st, t = sph_get_tuning(self.ctx)
        self._check(st)
        for k, v in kw.items():
            setattr(t, k, int(v))
        self._check(sph_set_tuning(self.ctx, t))

    def autotune(self, h0) -> dict:
        self._per_particle(h0, "h0")
        st, t = sph_autotune(self.ctx, h0.contiguous().data_ptr())
        self._check(st)
        return t.to_dict()

    def set_params(self, **params):
        self.params = make_params(**params)
        self._check(sph_set_params(self.ctx, self.params))

    def sort(self, pos, mass):
        torch = self._torch
        check_tensor(mass, "mass", torch.float64, ndim=1, cuda=False)
        n = int(mass.shape[0])
        check_tensor(pos, "pos", torch.float64, (3, n), cuda=False)
        for t, name in ((pos, "pos"), (mass, "mass")):
            check_tensor(t, name, t.dtype, device=self.device)
        pos = pos.contiguous()
        mass = mass.contiguous()
        self._pos, self._mass = pos, mass  # keep alive until the stream has used them
        self.n = 0
        self._check(sph_sort(self.ctx, n, pos.data_ptr(), mass.data_ptr()))
        self.n = n

    def solve(self, h0, out=None):
        torch = self._torch
        checks = [(h0, "h0", torch.float64)]
        if out is not None:
            checks += [(out[k], f"out['{k}']", dt) for k, dt in (("h", torch.float64), ("rho", torch.float64),
                                                                  ("count", torch.int32), ("nw", torch.float64))]
        for t, name, dt in checks:
            self._per_particle(t, name, dt, cuda=False)
        for t, name, dt in checks:
            self._per_particle(t, name, dt)
        if out is not None:
            for k in ("h", "rho", "count", "nw"):
                if not out[k].is_contiguous():
                    raise ValueError(f"out['{k}'] must be contiguous")
        h = h0.clone(memory_format=torch.contiguous_format) if out is None else out["h"].copy_(h0)
        rho = torch.empty_like(h) if out is None else out["rho"]
        count = torch.empty(h.shape[0], dtype=torch.int32, device=h.device) if out is None else out["count"]
        nw = torch.empty_like(h) if out is None else out["nw"]
        stats = SphStats()
        st = self._check(sph_density_solve(self.ctx, h.data_ptr(), rho.data_ptr(), count.data_ptr(),
                                           nw.data_ptr(), stats),
                         ok=(SPH_OK, SPH_ERR_NOT_CONVERGED, SPH_ERR_H_EXCEEDS_BOX))
        return {"h": h, "rho": rho, "count": count, "nw": nw, "status": st, "stats": stats.to_dict()}

    def knn(self, k, h0):
        """k-nearest-neighbour h (distance to the k-th nearest particle) and rho there; h0 is
        the starting search radius per particle."""
        torch = self._torch
        self._per_particle(h0, "h0")
        h = h0.clone(memory_format=torch.contiguous_format)
        rho = torch.empty_like(h)
        nw = torch.empty_like(h)
        count = torch.empty(h.shape[0], dtype=torch.int32, device=h.device)
        stats = SphStats()
        st = self._check(sph_knn_solve(self.ctx, int(k), h.data_ptr(), rho.data_ptr(), count.data_ptr(),
                                       nw.data_ptr(), stats),
                         ok=(SPH_OK, SPH_ERR_NOT_CONVERGED, SPH_ERR_H_EXCEEDS_BOX))
        return {"h": h, "rho": rho, "count": count, "nw": nw, "status": st, "stats": stats.to_dict()}

    def evaluate(self, h):
        torch = self._torch
        self._per_particle(h, "h")
        h = h.contiguous()
        rho = torch.empty_like(h)
        nw = torch.empty_like(h)
        dnw = torch.empty_like(h)
        count = torch.empty(h.shape[0], dtype=torch.int32, device=h.device)
        self._check(sph_density_eval(self.ctx, h.data_ptr(), rho.data_ptr(), count.data_ptr(),
                                     nw.data_ptr(), dnw.data_ptr()))
        return {"rho": rho, "nw": nw, "dnw": dnw, "count": count}

    def interact(self, h, vel):
        """Velocity mean, dispersion, divergence and curl over each particle's neighbours at its
        h (the further pair computations of the density loop).  vel: (3, n) float64.  Returns
        rho, vmean (3, n), sigma2, div, curl (3, n), count (int32) and the call's stats."""
        torch = self._torch
        vshape = (3, self.n) if self.n > 0 else None
        for cuda in (False, True):  # types and shapes of both first, then their device
            self._per_particle(h, "h", cuda=cuda)
            check_tensor(vel, "vel", torch.float64, vshape, self.device, ndim=2, cuda=cuda)
        h = h.contiguous()
        vel = vel.contiguous()
        rho = torch.empty_like(h)
        sigma2 = torch.empty_like(h)
        div = torch.empty_like(h)
        vmean = torch.empty_like(vel)
        curl = torch.empty_like(vel)
        count = torch.empty(h.shape[0], dtype=torch.int32, device=h.device)
        stats = SphStats()
        self._check(sph_interact(self.ctx, h.data_ptr(), vel.data_ptr(), rho.data_ptr(), vmean.data_ptr(),
                                 sigma2.data_ptr(), div.data_ptr(), curl.data_ptr(), count.data_ptr(), stats))
        return {"rho": rho, "vmean": vmean, "sigma2": sigma2, "div": div, "curl": curl, "count": count,
                "stats": stats.to_dict()}

    def neighbours(self, h, sample, max_nbr):
        """Neighbour sets of the sampled particles at fixed h (one density evaluation that also
        records them).  sample: int64 caller indices.  Returns nbr (n_sample, max_nbr) int32
        (row k: caller indices of sample k's neighbours, first nbr_count[k] entries valid, at
        most max_nbr), nbr_count (n_sample,) int32, and rho/count of every particle."""
        torch = self._torch
        self._per_particle(h, "h")
        check_tensor(sample, "sample", torch.int64, ndim=1, device=self.device)
        h = h.contiguous()
        sample = sample.contiguous()
        ns = int(sample.shape[0])
        nbr = torch.empty((ns, int(max_nbr)), dtype=torch.int32, device=h.device)
        nbr_count = torch.empty(ns, dtype=torch.int32, device=h.device)
        rho = torch.empty_like(h)
        count = torch.empty(h.shape[0], dtype=torch.int32, device=h.device)
        self._check(sph_neighbours_sampled(self.ctx, h.data_ptr(), ns, sample.data_ptr(), int(max_nbr),
                                           nbr.data_ptr(), nbr_count.data_ptr(), rho.data_ptr(),
                                           count.data_ptr()))
        return {"nbr": nbr, "nbr_count": nbr_count, "rho": rho, "count": count}

    def batch_solve(self, offsets, pos, mass, h0, nngb, tol):
        torch = self._torch
        check_tensor(offsets, "offsets", torch.int64, ndim=1, cuda=False)
        check_tensor(mass, "mass", torch.float64, ndim=1, cuda=False)
        n_all, g_all = int(mass.shape[0]), max(int(offsets.shape[0]) - 1, 0)
        check_tensor(pos, "pos", torch.float64, (3, n_all), cuda=False)
        check_tensor(h0, "h0", torch.float64, (n_all,), cuda=False)
        check_tensor(nngb, "nngb", torch.float64, (g_all,), cuda=False)
        check_tensor(tol, "tol", torch.float64, (g_all,), cuda=False)
        for t, name in ((offsets, "offsets"), (pos, "pos"), (mass, "mass"), (h0, "h0"), (nngb, "nngb"),
                        (tol, "tol")):
            check_tensor(t, name, t.dtype, device=self.device)
        self.n = 0  # the context now holds groups, not one sorted set
        offsets = offsets.contiguous()
        pos = pos.contiguous()
        mass = mass.contiguous()
        nngb = nngb.contiguous()
        tol = tol.contiguous()
        n = int(mass.shape[0])
        h = h0.clone(memory_format=torch.contiguous_format)
        rho = torch.empty_like(h)
        nw = torch.empty_like(h)
        count = torch.empty(n, dtype=torch.int32, device=h.device)
        stats = SphStats()
        st = self._check(sph_batch_solve(self.ctx, int(offsets.shape[0] - 1), offsets.data_ptr(),
                                         pos.data_ptr(), mass.data_ptr(), nngb.data_ptr(), tol.data_ptr(),
                                         h.data_ptr(), rho.data_ptr(), count.data_ptr(), nw.data_ptr(),
                                         stats),
                         ok=(SPH_OK, SPH_ERR_NOT_CONVERGED, SPH_ERR_H_EXCEEDS_BOX))
        return {"h": h, "rho": rho, "count": count, "nw": nw, "status": st, "stats": stats.to_dict()}
