"""Parity at the benchmark configurations' full sizes, on sampled outputs.

The GPU solves every particle; the FP64 oracle solves a random sample of targets against the
full particle set (the density is in gather form, so a target's solve depends only on the
positions and masses) by brute-force neighbour search, which needs no per-level grid over
tens of millions of particles.  Batched groups are independent, so a sample of whole groups
(always including the largest) is solved by the oracle and compared group by group.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1612_06090_gb300 import inputs
from tests.parity import check_solve, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1612_06090_gb300 import binding as B  # noqa: E402

DEV = torch.device("cuda:0")


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def _solve(wl, precision, h0=None, use_graph=False):
    s = B.Solver(wl.n, precision=precision, box=wl.box, nngb=wl.nngb, tol=wl.tol, use_graph=use_graph)
    s.sort(T(wl.pos), T(wl.mass))
    r = s.solve(T(wl.h0 if h0 is None else h0))
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    s.close()
    return out


def _sample_check(wl, g, n_samples, seed, precision, h0=None):
    rng = np.random.default_rng(seed)
    tg = np.sort(rng.choice(wl.n, size=n_samples, replace=False))
    start = wl.h0 if h0 is None else h0
    o = oracle.solve(wl.pos, wl.mass, start[tg], box=wl.box, nngb=wl.nngb, tol=wl.tol, targets=tg,
                     mode="brute")
    gs = {k: g[k][tg] for k in ("h", "rho", "count", "nw")}
    fp64 = precision == B.SPH_PREC_FP64
    return check_solve(wl.pos, wl.mass, wl.box, True, wl.nngb, wl.tol, gs, o, tg,
                       rtol=1e-12 if fp64 else 1e-5, delta=(1e-9 if fp64 else 1e-5) * wl.nngb,
                       max_mismatch_frac=0.002, count_exact=fp64, mode="brute"), o


@functools.lru_cache(maxsize=1)
def _c3():
    return inputs.make("c3")


def test_config3_lognormal_16M_sampled():
    wl = _c3()
    g = _solve(wl, B.SPH_PREC_FP32_KAHAN)
    assert g["status"] == B.SPH_OK
    _sample_check(wl, g, 96, 303, B.SPH_PREC_FP32_KAHAN)


def test_config5_clumps_67M_sampled_with_warm_start_snapshot():
    wl0 = inputs.make("c5", snapshot=0)
    g0 = _solve(wl0, B.SPH_PREC_FP32_KAHAN, use_graph=True)
    assert g0["status"] == B.SPH_OK
    _, o0 = _sample_check(wl0, g0, 48, 505, B.SPH_PREC_FP32_KAHAN)
    # snapshot 1 (every particle drifted by N(0, 1e-4^2)); each side warm-starts from its own
    # snapshot-0 answer
    wl1 = inputs.make("c5", snapshot=1)
    g1 = _solve(wl1, B.SPH_PREC_FP32_KAHAN, h0=g0["h"], use_graph=True)
    assert g1["status"] == B.SPH_OK
    assert g1["stats"]["passes"] < g0["stats"]["passes"]
    rng = np.random.default_rng(505)
    tg = np.sort(rng.choice(wl1.n, size=48, replace=False))
    o1 = oracle.solve(wl1.pos, wl1.mass, o0["h"], box=wl1.box, nngb=wl1.nngb, tol=wl1.tol, targets=tg,
                      mode="brute")
    gs = {k: g1[k][tg] for k in ("h", "rho", "count", "nw")}
    check_solve(wl1.pos, wl1.mass, wl1.box, True, wl1.nngb, wl1.tol, gs, o1, tg, rtol=1e-5,
                delta=1e-5 * wl1.nngb, max_mismatch_frac=0.002, count_exact=False, mode="brute")


@pytest.mark.parametrize("precision", [B.SPH_PREC_FP32_KAHAN])
def test_config4_batched_groups_sampled(precision):
    wl = inputs.make("c4")
    s = B.Solver(wl.n, precision=precision, use_graph=True)
    r = s.batch_solve(T(wl.offsets, torch.int64), T(wl.pos), T(wl.mass), T(wl.h0), T(wl.nngb), T(wl.tol))
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    s.close()
    assert g["status"] == B.SPH_OK
    assert np.all(np.abs(g["nw"] - 32.0) <= 1.0 + 1e-4)
    sizes = np.diff(wl.offsets)
    rng = np.random.default_rng(404)
    pick = set(rng.choice(wl.n_groups, size=40, replace=False).tolist())
    pick |= set(np.argsort(sizes)[-2:].tolist())  # the two largest groups
    for gi in sorted(pick):
        s0, e0 = int(wl.offsets[gi]), int(wl.offsets[gi + 1])
        o = oracle.solve(wl.pos[:, s0:e0], wl.mass[s0:e0], wl.h0[s0:e0], box=(0, 0, 0), periodic=False,
                         nngb=32.0, tol=1.0)
        assert np.all(o["status"] == 0)
        gs = {k: g[k][s0:e0] for k in ("h", "rho", "count", "nw")}
        check_solve(wl.pos[:, s0:e0], wl.mass[s0:e0], (0, 0, 0), False, 32.0, 1.0, gs, o,
                    np.arange(e0 - s0), rtol=1e-5, delta=1e-5 * 32, max_mismatch_frac=0.002,
                    count_exact=False)


def test_config3_lognormal_16M_knn_sampled():
    # the k-nearest-neighbour h at the paper's K = 295 on the 16.7M log-normal field (densities
    # spanning orders of magnitude), FP32 with estimated start radii, against the oracle's full
    # sort of every distance for sampled targets
    wl = _c3()
    s = B.Solver(wl.n, precision=B.SPH_PREC_FP32_KAHAN, box=wl.box)
    s.sort(T(wl.pos), T(wl.mass))
    r = s.knn(295, torch.zeros(wl.n, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    s.close()
    assert g["status"] == B.SPH_OK
    rng = np.random.default_rng(295)
    tg = np.sort(rng.choice(wl.n, size=48, replace=False))
    o = oracle.knn(wl.pos, wl.mass, 295, targets=tg, mode="brute")
    assert np.max(rel_err(g["h"][tg], o["h"])) <= 2e-6
    assert np.max(rel_err(g["rho"][tg], o["rho"])) <= 1e-5
    e = oracle.evaluate(wl.pos, wl.mass, g["h"][tg], targets=tg, near_rel=1e-6, mode="brute")
    assert np.all(np.abs(g["count"][tg].astype(np.int64) - e["count"]) <= e["near"])
