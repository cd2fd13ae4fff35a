"""FP64 CPU oracle for the SPH density / smoothing-length solve.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it; the CUDA library and its Python binding never import it.
It shares no code with the CUDA path.  The arithmetic lives in ``sph_oracle.c``
(plain C, FP64, OpenMP over the todo list); this module compiles it with gcc and
marshals numpy arrays through ctypes.

Functions
---------
w(q), mqdw(q)                M4 shape w(q) and -q w'(q)          (Eq. 1 kernel)
w_c6(q), mqdw_c6(q)          Wendland C6 shape (Sec. II-B kernel) and -q w'(q)
evaluate(...)                one fixed-h density evaluation      (Eq. 1, Listing 1)
solve(...)                   the h iteration on one particle set (Sec. IV-A, Listing 3)
h_update(...)                one step of that iteration's h update
batch_solve(...)             the same over independent non-periodic groups
knn(...)                     h = distance to the K-th nearest particle, rho at that h
                             (Sec. IV-D, the selection of the K nearest)
interact(...)                velocity mean, dispersion, divergence and curl over the same
                             neighbour sets (the further pair computations of Listing 1)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_PASSES = 64
STATUS_CONVERGED, STATUS_NOT_CONVERGED, STATUS_EXCEEDS_BOX = 0, 1, 2


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("passes", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("todo_per_pass", ctypes.c_int64 * MAX_PASSES),
        ("unconverged", ctypes.c_int64),
        ("exceeded", ctypes.c_int64),
        ("pair_evals", ctypes.c_int64),
    ]

    def to_dict(self):
        return {
            "passes": int(self.passes),
            "todo_per_pass": [int(v) for v in self.todo_per_pass[: max(0, min(self.passes, MAX_PASSES))]],
            "unconverged": int(self.unconverged),
            "exceeded": int(self.exceeded),
            "pair_evals": int(self.pair_evals),
        }


def build(force: bool = False) -> str:
    """Compile sph_oracle.c into liboracle.so next to it (gcc, OpenMP, no FP contraction)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                   "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_w.restype = ctypes.c_double
    lib.oracle_w.argtypes = [ctypes.c_double]
    lib.oracle_mqdw.restype = ctypes.c_double
    lib.oracle_mqdw.argtypes = [ctypes.c_double]
    lib.oracle_w_c6.restype = ctypes.c_double
    lib.oracle_w_c6.argtypes = [ctypes.c_double]
    lib.oracle_mqdw_c6.restype = ctypes.c_double
    lib.oracle_mqdw_c6.argtypes = [ctypes.c_double]
    lib.oracle_eval.restype = ctypes.c_int
    lib.oracle_eval.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int64, ip,
                                dp, ctypes.c_int, ctypes.c_double, dp, dp, dp, ip, ip, ctypes.c_int]
    lib.oracle_solve.restype = ctypes.c_int
    lib.oracle_solve.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_int64, ip, ctypes.c_int, dp,
                                 dp, dp, ip, i32p, ctypes.POINTER(OracleStats), ctypes.c_int]
    lib.oracle_batch_solve.restype = ctypes.c_int
    lib.oracle_batch_solve.argtypes = [ctypes.c_int64, ip, dp, dp, dp, dp, dp, dp, ctypes.c_int,
                                       ctypes.c_int, dp, dp, dp, ip, i32p,
                                       ctypes.POINTER(OracleStats), ctypes.c_int]
    lib.oracle_knn.restype = ctypes.c_int
    lib.oracle_knn.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int64, ip, ctypes.c_int, dp, dp, dp, ip, i32p, ctypes.c_int]
    lib.oracle_interact.restype = ctypes.c_int
    lib.oracle_interact.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int,
                                    ctypes.c_int64, ip, dp, ctypes.c_int, dp, dp, dp, dp, dp, ip, dp,
                                    ctypes.c_int]
    lib.oracle_h_update.restype = ctypes.c_double
    lib.oracle_h_update.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    dp, dp]
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_num_threads.argtypes = []
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    """OpenMP threads the oracle runs with (OMP_NUM_THREADS, else all cores)."""
    return int(_load().oracle_num_threads())


def w(q: float) -> float:
    """M4 shape function w(q); the kernel is W = 8 / (pi h^3) w(r/h)."""
    return float(_load().oracle_w(float(q)))


def mqdw(q: float) -> float:
    """-q w'(q); dN_w/dh = (32/3)(1/h) sum_j mqdw(q_j)."""
    return float(_load().oracle_mqdw(float(q)))


def w_c6(q: float) -> float:
    """Wendland C6 shape w(q); the kernel is W = 1365 / (64 pi h^3) w(r/h)."""
    return float(_load().oracle_w_c6(float(q)))


def mqdw_c6(q: float) -> float:
    """-q w'(q) of the Wendland C6 shape; dN_w/dh = (1365/48)(1/h) sum_j mqdw_c6(q_j)."""
    return float(_load().oracle_mqdw_c6(float(q)))


def h_update(h, nw, dnw, nngb, h_lo=0.0, h_hi=float("inf")):
    """One step of the h iteration from an evaluation (N_w, N_w') at h outside the band.

    h_lo / h_hi: the bracket before this evaluation (0 and +inf when unset).  Returns
    (next h, h_lo, h_hi) with the bracket updated by this evaluation.
    """
    lo = ctypes.c_double(h_lo)
    hi = ctypes.c_double(h_hi)
    hn = _load().oracle_h_update(float(h), float(nw), float(dnw), float(nngb), ctypes.byref(lo), ctypes.byref(hi))
    return float(hn), lo.value, hi.value


KERNELS = {"m4": 0, "wendland_c6": 1}


_MODES = {"grid": 0, "brute": 1}


def evaluate(pos, mass, h, box=(1.0, 1.0, 1.0), periodic=True, targets=None, mode="grid",
             near_rel=0.0, kernel="m4"):
    """One density evaluation at fixed smoothing lengths.

    pos: (3, N); mass: (N,); h: one value per target (targets=None: all N particles).
    Returns rho, nw (weighted count N_w), dnw (dN_w/dh), count (integer neighbours, self
    included) and, when near_rel > 0, near (pairs with |r - h| <= near_rel h).
    """
    lib = _load()
    pos = _f64(pos)
    mass = _f64(mass)
    n = mass.shape[0]
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.shape[0]
    h = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (nt,)))
    box = _f64(box)
    rho, nw, dnw = np.empty(nt), np.empty(nt), np.empty(nt)
    count = np.empty(nt, dtype=np.int64)
    near = np.zeros(nt, dtype=np.int64)
    x, y, z = (np.ascontiguousarray(pos[d]) for d in range(3))
    rc = lib.oracle_eval(n, _dp(x), _dp(y), _dp(z), _dp(mass), _dp(box), int(bool(periodic)),
                         nt if tg is not None else -1, _ip(tg) if tg is not None else None, _dp(h),
                         _MODES[mode], float(near_rel), _dp(rho), _dp(nw), _dp(dnw), _ip(count),
                         _ip(near), KERNELS[kernel])
    if rc != 0:
        raise MemoryError("oracle_eval failed to allocate")
    out = {"rho": rho, "nw": nw, "dnw": dnw, "count": count}
    if near_rel > 0.0:
        out["near"] = near
    return out


def solve(pos, mass, h0, box=(1.0, 1.0, 1.0), periodic=True, nngb=64.0, tol=2.0, max_iter=64,
          targets=None, mode="grid", kernel="m4"):
    """Run the smoothing-length iteration for the targets (None: all particles).

    Every particle contributes as a neighbour; only the targets are solved (the density
    is in gather form, so each target's solve depends only on positions and masses).
    Returns h, rho, nw, count, status (0 converged, 1 not converged, 2 h exceeds box) and
    the solve statistics.
    """
    lib = _load()
    pos = _f64(pos)
    mass = _f64(mass)
    n = mass.shape[0]
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.shape[0]
    h = np.array(np.broadcast_to(np.asarray(h0, dtype=np.float64), (nt,)), dtype=np.float64)
    box = _f64(box)
    rho, nw = np.empty(nt), np.empty(nt)
    count = np.empty(nt, dtype=np.int64)
    status = np.empty(nt, dtype=np.int32)
    st = OracleStats()
    x, y, z = (np.ascontiguousarray(pos[d]) for d in range(3))
    rc = lib.oracle_solve(n, _dp(x), _dp(y), _dp(z), _dp(mass), _dp(box), int(bool(periodic)),
                          float(nngb), float(tol), int(max_iter), nt if tg is not None else -1,
                          _ip(tg) if tg is not None else None, _MODES[mode], _dp(h), _dp(rho),
                          _dp(nw), _ip(count), _i32p(status), ctypes.byref(st), KERNELS[kernel])
    if rc != 0:
        raise MemoryError("oracle_solve failed to allocate")
    return {"h": h, "rho": rho, "nw": nw, "count": count, "status": status, "stats": st.to_dict()}


def batch_solve(offsets, pos, mass, h0, nngb, tol, max_iter=64, mode="grid", kernel="m4"):
    """The iteration over independent non-periodic groups (group g = [offsets[g], offsets[g+1]))."""
    lib = _load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    pos = _f64(pos)
    mass = _f64(mass)
    n = mass.shape[0]
    g = offsets.shape[0] - 1
    h = np.array(_f64(h0), dtype=np.float64)
    nngb = _f64(np.broadcast_to(np.asarray(nngb, dtype=np.float64), (g,)))
    tol = _f64(np.broadcast_to(np.asarray(tol, dtype=np.float64), (g,)))
    rho, nw = np.empty(n), np.empty(n)
    count = np.empty(n, dtype=np.int64)
    status = np.empty(n, dtype=np.int32)
    st = OracleStats()
    x, y, z = (np.ascontiguousarray(pos[d]) for d in range(3))
    rc = lib.oracle_batch_solve(g, _ip(offsets), _dp(x), _dp(y), _dp(z), _dp(mass), _dp(nngb),
                                _dp(tol), int(max_iter), _MODES[mode], _dp(h), _dp(rho), _dp(nw),
                                _ip(count), _i32p(status), ctypes.byref(st), KERNELS[kernel])
    if rc != 0:
        raise MemoryError("oracle_batch_solve failed to allocate")
    return {"h": h, "rho": rho, "nw": nw, "count": count, "status": status, "stats": st.to_dict()}


def knn(pos, mass, k, box=(1.0, 1.0, 1.0), periodic=True, targets=None, mode="grid", kernel="m4"):
    """k-nearest-neighbour smoothing lengths for the targets (None: all particles).

    h = distance to the k-th nearest particle (the particle itself is the first, at r = 0),
    every squared distance formed as in the density pairs and the list sorted; rho, nw and
    count (#{r < h}, self included) are the fixed-h evaluation at that h.  status 0, or 2
    when a periodic h reaches min(box)/2 (no density then).  Needs 2 <= k <= n.
    """
    lib = _load()
    pos = _f64(pos)
    mass = _f64(mass)
    n = mass.shape[0]
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.shape[0]
    box = _f64(box)
    h, rho, nw = np.empty(nt), np.empty(nt), np.empty(nt)
    count = np.empty(nt, dtype=np.int64)
    status = np.empty(nt, dtype=np.int32)
    x, y, z = (np.ascontiguousarray(pos[d]) for d in range(3))
    rc = lib.oracle_knn(n, _dp(x), _dp(y), _dp(z), _dp(mass), _dp(box), int(bool(periodic)), int(k),
                        nt if tg is not None else -1, _ip(tg) if tg is not None else None,
                        _MODES[mode], _dp(h), _dp(rho), _dp(nw), _ip(count), _i32p(status),
                        KERNELS[kernel])
    if rc == -2:
        raise ValueError("k must lie in [2, n]")
    if rc != 0:
        raise MemoryError("oracle_knn failed to allocate")
    return {"h": h, "rho": rho, "nw": nw, "count": count, "status": status}


def interact(pos, mass, vel, h, box=(1.0, 1.0, 1.0), periodic=True, targets=None, mode="grid",
             kernel="m4"):
    """Velocity-field estimates over each target's neighbours at its h (gather form).

    pos, vel: (3, N); mass: (N,); h: one value per target (targets=None: all N particles).
    Returns rho (Eq. 1), vmean (3, T) = (1/rho) sum m W v_j, sigma2 = (1/rho) sum m W
    |v_j - vmean|^2, div = (1/rho) sum m (v_j - v_i) . grad_i W, curl (3, T) = (1/rho) sum
    m (v_i - v_j) x grad_i W, count (#{r < h}, self included) and the error scales vscale2
    ((1/rho) sum m W |v_j - v_i|^2), gabs ((1/rho) sum m |grad W| |v_j - v_i|), gnorm ((1/rho)
    sum m |grad W|) and vmax (largest velocity component magnitude among the neighbours).
    """
    lib = _load()
    pos = _f64(pos)
    vel = _f64(vel)
    mass = _f64(mass)
    n = mass.shape[0]
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tg is None else tg.shape[0]
    h = _f64(np.broadcast_to(np.asarray(h, dtype=np.float64), (nt,)))
    box = _f64(box)
    rho, sigma2, div = np.empty(nt), np.empty(nt), np.empty(nt)
    vmean, curl = np.empty((3, nt)), np.empty((3, nt))
    count = np.empty(nt, dtype=np.int64)
    scales = np.empty((4, nt))
    x, y, z = (np.ascontiguousarray(pos[d]) for d in range(3))
    vx, vy, vz = (np.ascontiguousarray(vel[d]) for d in range(3))
    rc = lib.oracle_interact(n, _dp(x), _dp(y), _dp(z), _dp(mass), _dp(vx), _dp(vy), _dp(vz), _dp(box),
                             int(bool(periodic)), nt if tg is not None else -1,
                             _ip(tg) if tg is not None else None, _dp(h), _MODES[mode], _dp(rho),
                             _dp(vmean), _dp(sigma2), _dp(div), _dp(curl), _ip(count), _dp(scales),
                             KERNELS[kernel])
    if rc != 0:
        raise MemoryError("oracle_interact failed to allocate")
    return {"rho": rho, "vmean": vmean, "sigma2": sigma2, "div": div, "curl": curl, "count": count,
            "vscale2": scales[0], "gabs": scales[1], "gnorm": scales[2], "vmax": scales[3]}
