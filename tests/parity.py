"""Helpers that compare CUDA results with the FP64 oracle.

The solve is an iteration whose answer is not unique: any h with |N_w - Nngb| <= tol is a
valid answer, so the two sides agree element by element only while they take the same
decisions.  Both start from the same h0 and follow the same update rule, so they do,
except for particles whose N_w lands within rounding of a band edge.  For those the GPU
answer is checked instead: the oracle, evaluated at the GPU's h, must put N_w in the band
and reproduce the GPU's density.
"""
import numpy as np

import oracle


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def check_eval(gpu, orc, rtol, count_exact=True, near=None, dnw_rtol=None):
    """Fixed-h evaluation: rho, N_w, dN_w/dh within rtol; counts exact or within the pairs
    the oracle finds at |r - h| <= eps h (`near`)."""
    assert np.max(rel_err(gpu["rho"], orc["rho"])) <= rtol, np.max(rel_err(gpu["rho"], orc["rho"]))
    assert np.max(rel_err(gpu["nw"], orc["nw"])) <= rtol, np.max(rel_err(gpu["nw"], orc["nw"]))
    if "dnw" in gpu and "dnw" in orc:
        r = dnw_rtol if dnw_rtol is not None else rtol
        scale = np.maximum(np.abs(orc["dnw"]), np.abs(orc["nw"]) / np.maximum(gpu.get("h", 1.0), 1e-300) * 1e-3)
        err = np.abs(np.asarray(gpu["dnw"]) - orc["dnw"]) / np.maximum(scale, 1e-300)
        assert np.max(err) <= r, np.max(err)
    dc = np.abs(np.asarray(gpu["count"], dtype=np.int64) - orc["count"])
    if count_exact:
        assert np.all(dc == 0), int(dc.max())
    else:
        assert near is not None
        assert np.all(dc <= near), (dc[dc > near][:5], near[dc > near][:5])


def check_solve(pos, mass, box, periodic, nngb, tol, gpu, orc, targets, rtol, delta,
                max_mismatch_frac, count_exact=True, mode="grid", kernel=None):
    """Compare a GPU solve with an oracle solve of the same targets (see module docstring).

    gpu: numpy dict of h, rho, count, nw for the targets; orc: oracle.solve output for them.
    Returns the fraction of particles checked through the band-edge route."""
    assert np.all(orc["status"] == 0), "the oracle did not converge"
    eh = rel_err(gpu["h"], orc["h"])
    er = rel_err(gpu["rho"], orc["rho"])
    mism = (eh > rtol) | (er > rtol)
    frac = float(np.mean(mism))
    ok = ~mism
    if count_exact:
        d = np.asarray(gpu["count"], dtype=np.int64)[ok] - orc["count"][ok]
        assert np.all(d == 0), int(np.abs(d).max())
    else:
        e = oracle.evaluate(pos, mass, np.asarray(gpu["h"])[ok], box=box, periodic=periodic,
                            targets=np.asarray(targets)[ok], near_rel=1e-6, mode=mode,
                            kernel=kernel or "m4")
        d = np.abs(np.asarray(gpu["count"], dtype=np.int64)[ok] - e["count"])
        assert np.all(d <= e["near"])
    if mism.any():
        idx = np.flatnonzero(mism)
        e = oracle.evaluate(pos, mass, np.asarray(gpu["h"])[idx], box=box, periodic=periodic,
                            targets=np.asarray(targets)[idx], near_rel=1e-6, mode=mode,
                            kernel=kernel or "m4")
        assert np.all(np.abs(e["nw"] - nngb) <= tol + delta), np.abs(e["nw"] - nngb).max()
        assert np.max(rel_err(np.asarray(gpu["rho"])[idx], e["rho"])) <= rtol
    assert frac <= max_mismatch_frac, frac
    # every GPU answer lies in the band
    assert np.all(np.abs(np.asarray(gpu["nw"]) - nngb) <= tol + delta)
    return frac
