"""Cached neighbour lists (params.list_entries > 0): parity and equivalence on the GPU.

A search records, for every target, the particles within (1 + margin) h; a later pass of the
same solve whose h stays within that radius evaluates the list instead of searching.  The list
holds every particle the search would test within the new h, so:
  - FP64 mode forms every list pair exactly as the FP64 formulae are written: counts equal the
    oracle's, rho/N_w/h agree to 1e-12, and the pass count, per-pass todo counts and in-h pair
    count equal the oracle's;
  - FP32 mode forms list offsets from exact fixed-point differences: the usual FP32 bounds hold
    (1e-5, counts within the pairs 1e-6 h from the boundary, at most 0.2 % band-edge particles);
  - the CUDA-graph loop gives bitwise the host loop's results, and statistics show that lists
    were used (list_evals > 0) and that the first pass searched every target.
"""
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

FP64, FP32 = B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN
DEV = torch.device("cuda:0")


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def solve(wl, precision, list_entries=192, use_graph=False, h0=None, margin=None, **kw):
    s = B.Solver(wl.n, precision=precision, box=wl.box, nngb=wl.nngb, tol=wl.tol,
                 list_entries=list_entries, use_graph=use_graph, **kw)
    if margin is not None:
        s.set_tuning(list_margin_pct=margin)
    s.sort(T(wl.pos), T(wl.mass))
    r = s.solve(T(wl.h0 if h0 is None else h0))
    torch.cuda.synchronize()
    out = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    s.close()
    return out


def test_fp64_lists_match_the_oracle_exactly_config1():
    wl = inputs.make("c1")
    g = solve(wl, FP64)
    assert g["status"] == B.SPH_OK
    assert g["stats"]["list_evals"] > 0
    o = oracle.solve(wl.pos, wl.mass, wl.h0)
    check_solve(wl.pos, wl.mass, wl.box, True, 64.0, 2.0, g, o, np.arange(wl.n), rtol=1e-12,
                delta=1e-9 * 64, max_mismatch_frac=1e-3, count_exact=True)
    assert g["stats"]["passes"] == o["stats"]["passes"]
    assert g["stats"]["todo_per_pass"] == o["stats"]["todo_per_pass"]
    assert g["stats"]["pair_evals"] == o["stats"]["pair_evals"]


@pytest.mark.parametrize("margin", [5, 10, 30])
def test_fp32_lists_against_the_oracle_config1(margin):
    wl = inputs.make("c1")
    g = solve(wl, FP32, margin=margin)
    assert g["status"] == B.SPH_OK
    assert g["stats"]["list_evals"] > 0
    o = oracle.solve(wl.pos, wl.mass, wl.h0)
    check_solve(wl.pos, wl.mass, wl.box, True, 64.0, 2.0, g, o, np.arange(wl.n), rtol=1e-5,
                delta=1e-5 * 64, max_mismatch_frac=0.002, count_exact=False)


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_lists_on_the_cluster_set_sampled(precision):
    """1,048,576 Plummer-cluster particles from the common h0: the sphere cores start with
    thousands of candidates (no list fits) and find lists as h shrinks."""
    wl = inputs.make("c2")
    g = solve(wl, precision)
    assert g["status"] == B.SPH_OK
    assert g["stats"]["list_evals"] > 0
    rng = np.random.default_rng(2024)
    tg = np.sort(rng.choice(wl.n, size=1500, replace=False))
    o = oracle.solve(wl.pos, wl.mass, wl.h0[tg], targets=tg)
    gs = {k: g[k][tg] for k in ("h", "rho", "count", "nw")}
    fp64 = precision == FP64
    check_solve(wl.pos, wl.mass, wl.box, True, 64.0, 2.0, gs, o, tg, rtol=1e-12 if fp64 else 1e-5,
                delta=(1e-9 if fp64 else 1e-5) * 64, max_mismatch_frac=0.002, count_exact=fp64)


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_graph_loop_with_lists_matches_host_loop(precision):
    wl = inputs.make("c2", n=1 << 16)
    a = solve(wl, precision, use_graph=False)
    b = solve(wl, precision, use_graph=True)
    for k in ("h", "rho", "nw", "count"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["stats"]["todo_per_pass"] == b["stats"]["todo_per_pass"]
    assert a["stats"]["list_evals"] == b["stats"]["list_evals"] > 0


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_lists_change_nothing_beyond_rounding(precision):
    wl = inputs.make("c2", n=1 << 17)
    a = solve(wl, precision, list_entries=0)
    b = solve(wl, precision)
    assert a["stats"]["list_evals"] == 0 < b["stats"]["list_evals"]
    tol = 1e-12 if precision == FP64 else 1e-5
    same = rel_err(b["h"], a["h"]) <= tol
    assert same.mean() > 0.999
    assert np.max(rel_err(b["rho"][same], a["rho"][same])) <= tol
    if precision == FP64:
        np.testing.assert_array_equal(a["count"][same], b["count"][same])


def test_lists_too_short_fall_back_to_the_search():
    # 16 entries cannot hold a 64-neighbour list with its margin: every pass searches
    wl = inputs.make("c1")
    g = solve(wl, FP64, list_entries=16)
    assert g["status"] == B.SPH_OK
    assert g["stats"]["list_evals"] == 0
    o = oracle.solve(wl.pos, wl.mass, wl.h0)
    np.testing.assert_array_equal(g["count"], o["count"])
    assert np.max(rel_err(g["rho"], o["rho"])) <= 1e-12


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_batch_with_lists_matches_oracle(precision):
    wl = inputs.plummer_groups(n_groups=60, nmin=32, nmax=20000, seed=31)
    s = B.Solver(wl.n, precision=precision, list_entries=128)
    r = s.batch_solve(T(wl.offsets, torch.int64), T(wl.pos), T(wl.mass), T(wl.h0), T(wl.nngb), T(wl.tol))
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    s.close()
    assert g["status"] == B.SPH_OK
    assert g["stats"]["list_evals"] > 0
    o = oracle.batch_solve(wl.offsets, wl.pos, wl.mass, wl.h0, wl.nngb, wl.tol)
    rtol = 1e-12 if precision == FP64 else 1e-5
    mism = (rel_err(g["h"], o["h"]) > rtol) | (rel_err(g["rho"], o["rho"]) > rtol)
    assert mism.mean() <= 0.002
    if precision == FP64:
        np.testing.assert_array_equal(g["count"][~mism], o["count"][~mism])
    assert np.all(np.abs(g["nw"] - 32.0) <= 1.0 + 1e-4)


def test_list_entries_is_fixed_per_context():
    s = B.Solver(100, precision=FP32, list_entries=64)
    with pytest.raises(B.SphError) as e:
        s.set_params(list_entries=128)
    assert e.value.status == B.SPH_ERR_INVALID_ARG
    s.set_params(list_entries=64, tol=3.0)
    s.close()
