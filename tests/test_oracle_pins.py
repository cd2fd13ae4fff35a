"""Pins of the FP64 oracle against mathematics, independent of the oracle's own code.

Each test fixes a fact the method (Eq. 1 with the M4 kernel, the h iteration of
Sec. IV-A) must satisfy, chosen so that a plausible slip in the oracle (a wrong
coefficient, a dropped self term, a wrong periodic image, a sign error in the update)
fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
from paper_1612_06090_gb300 import inputs
from tests import brute

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# --------------------------------------------------------------------------------------
# Kernel shape: these properties determine the M4 cubic B-spline uniquely
# --------------------------------------------------------------------------------------

def test_kernel_value_at_origin_and_support():
    assert oracle.w(0.0) == 1.0
    for q in (1.0, 1.0 + 1e-12, 1.5, 7.0):
        assert oracle.w(q) == 0.0
        assert oracle.mqdw(q) == 0.0


def test_kernel_normalisation_is_one():
    # int W d^3r = (8/pi) * 4 pi * int_0^1 q^2 w(q) dq = 32 int_0^1 q^2 w(q) dq = 1
    val, err = integrate.quad(lambda q: q * q * oracle.w(q), 0.0, 1.0, points=[0.5],
                              epsabs=1e-15, epsrel=1e-14)
    assert abs(32.0 * val - 1.0) < 1e-12


def _derivs(f, q, eps):
    d1 = (f(q + eps) - f(q - eps)) / (2 * eps)
    d2 = (f(q + eps) - 2 * f(q) + f(q - eps)) / (eps * eps)
    return d1, d2


def test_kernel_is_c2_spline_with_knot_at_half():
    # one-sided values and derivatives agree at q = 1/2 (C^2), and vanish at q = 1
    eps = 1e-5
    left = [oracle.w(0.5 - k * eps) for k in range(3)]
    right = [oracle.w(0.5 + k * eps) for k in range(3)]
    # value continuity
    assert abs(left[0] - right[1]) < 1e-4
    # first derivative from each side
    dl = (left[0] - left[1]) / eps
    dr = (right[1] - left[0]) / eps
    assert abs(dl - dr) < 1e-3
    # second derivative from each side
    d2l = (left[0] - 2 * left[1] + left[2]) / eps**2
    d2r = (right[2] - 2 * right[1] + left[0]) / eps**2
    assert abs(d2l - d2r) < 1e-2 * max(1.0, abs(d2l))
    # w, w', w'' all go to zero at the edge of the support
    q = 1.0 - 1e-4
    assert abs(oracle.w(q)) < 1e-11
    d1, d2 = _derivs(oracle.w, 1.0 - 2e-3, 1e-4)
    assert abs(d1) < 1e-4 and abs(d2) < 0.1
    # even kernel: w'(0) = 0
    assert abs((oracle.w(1e-6) - oracle.w(0.0)) / 1e-6) < 1e-4


def test_kernel_piece_values():
    # The C^2 cubic spline with w(0)=1, w'(0)=0 and zero C^2 contact at q=1 has
    # w(1/2) = 1/4; the same conditions fix w(1/4) = 0.71875 and w(3/4) = 1/32.
    assert oracle.w(0.5) == pytest.approx(0.25, abs=1e-15)
    assert oracle.w(0.25) == pytest.approx(0.71875, abs=1e-15)
    assert oracle.w(0.75) == pytest.approx(1.0 / 32.0, abs=1e-15)


def test_mqdw_is_minus_q_times_derivative_of_w():
    for q in np.linspace(0.01, 0.99, 97):
        if abs(q - 0.5) < 2e-6:
            continue
        d1, _ = _derivs(oracle.w, q, 1e-6)
        assert oracle.mqdw(q) == pytest.approx(-q * d1, rel=1e-7, abs=1e-9)


# --------------------------------------------------------------------------------------
# Neighbour search and sums: brute force, lattice, closed forms
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["grid", "brute"])
def test_fixed_h_matches_numpy_brute_force(mode):
    wl = inputs.make("c1")
    rng = np.random.default_rng(11)
    h = wl.h0 * rng.uniform(0.5, 2.0, size=wl.n)
    o = oracle.evaluate(wl.pos, wl.mass, h, mode=mode)
    b = brute.evaluate(wl.pos, wl.mass, h)
    np.testing.assert_array_equal(o["count"], b["count"])
    np.testing.assert_allclose(o["rho"], b["rho"], rtol=1e-13)
    np.testing.assert_allclose(o["nw"], b["nw"], rtol=1e-13)
    np.testing.assert_allclose(o["dnw"], b["dnw"], rtol=1e-12)


def test_adversarial_positions_on_cell_faces_and_box_edges():
    # particles exactly on bucket faces of several grid levels, at the box corner and
    # across the periodic seam
    rng = np.random.default_rng(5)
    k = rng.integers(0, 64, size=(3, 600))
    pos = k / 64.0
    pos[:, :8] = np.array([[0, 0, 0], [1 - 2**-30, 0, 0], [0, 1 - 2**-30, 0],
                           [0, 0, 1 - 2**-30], [0.5, 0.5, 0.5], [0.25, 0.75, 0.0],
                           [1 - 2**-40, 1 - 2**-40, 1 - 2**-40], [2**-40, 0.5, 0.5]]).T
    mass = rng.uniform(0.5, 1.5, size=600)
    h = np.full(600, 0.125)
    h[::3] = 0.0625
    h[1::3] = 3.0 / 64.0 + 1e-12
    o = oracle.evaluate(pos, mass, h)
    b = brute.evaluate(pos, mass, h)
    np.testing.assert_array_equal(o["count"], b["count"])
    np.testing.assert_allclose(o["rho"], b["rho"], rtol=1e-13)


def test_non_cubic_periodic_box_matches_brute_force():
    # box lengths differ per axis: each axis wraps with its own length
    box = (1.0, 0.5, 2.0)
    rng = np.random.default_rng(12)
    pos = rng.uniform(0.0, 1.0, size=(3, 1500)) * np.array(box)[:, None]
    mass = rng.uniform(0.5, 1.5, size=1500)
    h = rng.uniform(0.05, 0.24, size=1500)
    o = oracle.evaluate(pos, mass, h, box=box)
    b = brute.evaluate(pos, mass, h, box=box)
    np.testing.assert_array_equal(o["count"], b["count"])
    np.testing.assert_allclose(o["rho"], b["rho"], rtol=1e-13)
    np.testing.assert_allclose(o["dnw"], b["dnw"], rtol=1e-12)
    spatial = pytest.importorskip("scipy.spatial")
    tg = np.arange(0, 1500, 11)
    r = oracle.knn(pos, mass, 40, box=box, targets=tg)
    d, _ = spatial.cKDTree(pos.T, boxsize=np.array(box)).query(pos.T[tg], k=40)
    np.testing.assert_allclose(r["h"], d[:, -1], rtol=1e-14)


def test_non_periodic_matches_brute_force():
    rng = np.random.default_rng(8)
    pos = rng.normal(0.0, 3.0, size=(3, 700))
    mass = rng.uniform(0.1, 1.0, size=700)
    h = rng.uniform(0.5, 6.0, size=700)
    o = oracle.evaluate(pos, mass, h, periodic=False, box=(0, 0, 0))
    b = brute.evaluate(pos, mass, h, periodic=False)
    np.testing.assert_array_equal(o["count"], b["count"])
    np.testing.assert_allclose(o["rho"], b["rho"], rtol=1e-13)
    np.testing.assert_allclose(o["dnw"], b["dnw"], rtol=1e-12)


def _lattice16():
    g = (np.arange(16) + 0.5) / 16.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()]), np.full(4096, 1.0 / 4096)


def test_uniform_lattice_density_matches_lattice_sum():
    gold = json.load(open(os.path.join(GOLDEN, "lattice16.json")))
    pos, mass = _lattice16()
    o = oracle.evaluate(pos, mass, np.full(4096, gold["h0"]))
    # every particle sees the same lattice: identical values up to summation order
    assert np.all(o["count"] == gold["count_at_h0"])
    np.testing.assert_allclose(o["rho"], gold["rho_at_h0"], rtol=1e-13)
    np.testing.assert_allclose(o["nw"], gold["nw_at_h0"], rtol=1e-13)
    # kernel interpolation of a uniform density recovers it to ~0.1 % at 64 neighbours
    assert abs(o["rho"].mean() - 1.0) < 2e-3


def test_uniform_lattice_converges_at_pass_zero():
    gold = json.load(open(os.path.join(GOLDEN, "lattice16.json")))
    pos, mass = _lattice16()
    r = oracle.solve(pos, mass, np.full(4096, gold["h0"]), nngb=64.0, tol=2.0)
    assert r["stats"]["passes"] == 1
    assert np.all(r["status"] == 0)
    assert np.all(r["h"] == gold["h0"])


def test_lattice_root_by_refined_solve():
    gold = json.load(open(os.path.join(GOLDEN, "lattice16.json")))
    pos, mass = _lattice16()
    r = oracle.solve(pos, mass, np.full(4096, gold["h0"]), nngb=64.0, tol=1e-10, max_iter=64)
    assert np.all(r["status"] == 0)
    np.testing.assert_allclose(r["h"], gold["root_nw_64"], rtol=1e-12)


def test_two_particles_closed_form_across_periodic_seam():
    r = 0.02
    pos = np.array([[0.01, 0.99], [0.5, 0.5], [0.5, 0.5]])
    mass = np.array([1.0, 3.0])
    h = 0.05
    o = oracle.evaluate(pos, mass, np.array([h, h]))
    q = r / h
    # W = 8/(pi h^3) w; the self term has w(0) = 1
    w_q = 1.0 - 6.0 * q**2 + 6.0 * q**3  # q = 0.4 lies on the inner piece
    norm = 8.0 / (math.pi * h**3)
    assert o["count"].tolist() == [2, 2]
    assert o["rho"][0] == pytest.approx(norm * (1.0 * 1.0 + 3.0 * w_q), rel=1e-14)
    assert o["rho"][1] == pytest.approx(norm * (3.0 * 1.0 + 1.0 * w_q), rel=1e-14)
    assert o["nw"][0] == pytest.approx(32.0 / 3.0 * (1.0 + w_q), rel=1e-14)


def test_single_particle_self_floor():
    pos = np.array([[0.3], [0.4], [0.5]])
    o = oracle.evaluate(pos, np.array([2.0]), np.array([0.1]))
    assert o["count"][0] == 1
    assert o["nw"][0] == pytest.approx(32.0 / 3.0, rel=1e-15)
    assert o["rho"][0] == pytest.approx(2.0 * 8.0 / (math.pi * 0.1**3), rel=1e-14)
    assert o["dnw"][0] == 0.0


def test_dnw_matches_finite_difference_of_nw():
    wl = inputs.make("c1")
    rng = np.random.default_rng(3)
    tg = rng.choice(wl.n, size=64, replace=False)
    h = wl.h0[tg] * rng.uniform(0.8, 1.3, size=64)
    eps = 1e-7
    o = oracle.evaluate(wl.pos, wl.mass, h, targets=tg)
    # away from neighbour-set changes N_w is smooth; C^1 across them because w(1) = w'(1) = 0
    up = oracle.evaluate(wl.pos, wl.mass, h * (1 + eps), targets=tg)
    dn = oracle.evaluate(wl.pos, wl.mass, h * (1 - eps), targets=tg)
    fd = (up["nw"] - dn["nw"]) / (2 * eps * h)
    np.testing.assert_allclose(o["dnw"], fd, rtol=2e-5)


def test_nw_is_non_decreasing_in_h():
    wl = inputs.make("c1")
    tg = np.arange(0, wl.n, 97)
    prev = None
    for f in np.linspace(0.3, 2.5, 40):
        o = oracle.evaluate(wl.pos, wl.mass, wl.h0[tg] * f, targets=tg)
        if prev is not None:
            assert np.all(o["nw"] >= prev - 1e-12)
        prev = o["nw"]


def test_rho_and_nw_relation_for_equal_masses():
    # N_w = (4 pi / 3) h^3 rho / m when every mass is m
    wl = inputs.make("c1")
    o = oracle.evaluate(wl.pos, wl.mass, wl.h0)
    np.testing.assert_allclose(o["nw"], 4.0 * math.pi / 3.0 * wl.h0**3 * o["rho"] / wl.mass, rtol=1e-13)


# --------------------------------------------------------------------------------------
# The h iteration
# --------------------------------------------------------------------------------------

def test_solve_config1_all_converged_in_band_and_unique_root_bracketed():
    wl = inputs.make("c1")
    r = oracle.solve(wl.pos, wl.mass, wl.h0, nngb=64.0, tol=2.0)
    assert np.all(r["status"] == 0)
    assert np.all(np.abs(r["nw"] - 64.0) <= 2.0)
    # outputs describe the final evaluation
    o = oracle.evaluate(wl.pos, wl.mass, r["h"])
    np.testing.assert_array_equal(o["count"], r["count"])
    np.testing.assert_allclose(o["rho"], r["rho"], rtol=1e-14)
    # the solution lies between the roots of N_w = 62 and N_w = 66 (N_w is monotone)
    rng = np.random.default_rng(0)
    for i in rng.choice(wl.n, size=6, replace=False):
        f = lambda hh, t: oracle.evaluate(wl.pos, wl.mass, np.array([hh]), targets=np.array([i]))["nw"][0] - t
        lo = optimize.brentq(f, 0.3 * wl.h0[i], 3 * wl.h0[i], args=(62.0,), xtol=1e-15)
        hi = optimize.brentq(f, 0.3 * wl.h0[i], 3 * wl.h0[i], args=(66.0,), xtol=1e-15)
        assert lo - 1e-12 <= r["h"][i] <= hi + 1e-12


def test_refined_solve_matches_independent_root_finder():
    wl = inputs.make("c1")
    tg = np.arange(0, wl.n, 411)
    r = oracle.solve(wl.pos, wl.mass, wl.h0[tg], nngb=64.0, tol=1e-9, targets=tg)
    assert np.all(r["status"] == 0)
    for k, i in enumerate(tg):
        f = lambda hh: oracle.evaluate(wl.pos, wl.mass, np.array([hh]), targets=np.array([i]))["nw"][0] - 64.0
        root = optimize.brentq(f, 0.3 * wl.h0[i], 3 * wl.h0[i], xtol=1e-16, rtol=1e-15)
        assert r["h"][k] == pytest.approx(root, rel=1e-9)


def test_permutation_invariance():
    wl = inputs.make("c1")
    r = oracle.solve(wl.pos, wl.mass, wl.h0)
    perm = np.random.default_rng(9).permutation(wl.n)
    rp = oracle.solve(wl.pos[:, perm], wl.mass[perm], wl.h0[perm])
    np.testing.assert_allclose(rp["h"], r["h"][perm], rtol=1e-13)
    np.testing.assert_allclose(rp["rho"], r["rho"][perm], rtol=1e-13)
    np.testing.assert_array_equal(rp["count"], r["count"][perm])


def test_periodic_translation_invariance():
    wl = inputs.make("c1")
    r = oracle.solve(wl.pos, wl.mass, wl.h0)
    shift = np.array([0.3141592653589793, 0.7, 0.123456789])[:, None]
    pos = np.mod(wl.pos + shift, 1.0)
    pos[pos >= 1.0] = 0.0
    rs = oracle.solve(pos, wl.mass, wl.h0)
    np.testing.assert_allclose(rs["rho"], r["rho"], rtol=1e-10)
    np.testing.assert_allclose(rs["h"], r["h"], rtol=1e-10)


def test_mass_scaling():
    wl = inputs.make("c1")
    r = oracle.solve(wl.pos, wl.mass, wl.h0)
    r2 = oracle.solve(wl.pos, 4.0 * wl.mass, wl.h0)
    np.testing.assert_array_equal(r2["h"], r["h"])  # N_w does not depend on the masses
    np.testing.assert_array_equal(r2["rho"], 4.0 * r["rho"])  # exact: power-of-two scale


def test_single_particle_grows_until_box_limit():
    # N_w = 32/3 for every h and dN_w/dh = 0: Newton is never taken and h grows by
    # 2^(1/3) per pass until the next h would reach half the box.
    pos = np.array([[0.2], [0.2], [0.2]])
    h0 = 0.01
    r = oracle.solve(pos, np.array([1.0]), np.array([h0]), nngb=64.0, tol=2.0)
    assert r["status"][0] == oracle.STATUS_EXCEEDS_BOX
    k = r["stats"]["passes"] - 1
    h = h0
    for _ in range(k):
        h = h * 1.2599210498948732
    assert r["h"][0] == h
    assert h * 1.2599210498948732 >= 0.5 and h < 0.5
    assert r["rho"][0] == pytest.approx(8.0 / (math.pi * h**3), rel=1e-14)


def test_coincident_cluster_shrinks_until_pass_limit():
    # 100 coincident particles: N_w = 100 * 32/3 > Nngb for every h and dN_w/dh = 0,
    # so h falls by 2^(1/3) per pass and the solve stops after max_iter passes.
    pos = np.full((3, 100), 0.5)
    r = oracle.solve(pos, np.full(100, 0.01), np.full(100, 0.1), nngb=64.0, tol=2.0, max_iter=10)
    assert np.all(r["status"] == oracle.STATUS_NOT_CONVERGED)
    assert r["stats"]["passes"] == 10
    h = 0.1
    for _ in range(9):
        h = h / 1.2599210498948732
    assert np.all(r["h"] == h)
    assert r["stats"]["todo_per_pass"] == [100] * 10


def test_two_particle_root_closed_form():
    # N_w(h) = (32/3)(1 + w(r/h)) for h > r: with Nngb = 16 the root has w(q*) = 1/2,
    # i.e. 6 q^3 - 6 q^2 + 1/2 = 0 on the inner piece.
    r_sep = 0.05
    pos = np.array([[0.4, 0.4 + r_sep], [0.5, 0.5], [0.5, 0.5]])
    roots = np.roots([6.0, -6.0, 0.0, 0.5])
    qs = [x.real for x in roots if abs(x.imag) < 1e-12 and 0 < x.real <= 0.5]
    assert len(qs) == 1
    h_star = r_sep / qs[0]
    res = oracle.solve(pos, np.array([1.0, 1.0]), np.array([0.03, 0.2]), nngb=16.0, tol=1e-9)
    assert np.all(res["status"] == 0)
    np.testing.assert_allclose(res["h"], h_star, rtol=1e-9)


GROWTH = 1.2599210498948732  # 2^(1/3) as the double literal of the update rule


def _trajectory(pos, mass, h0, targets, passes, **kw):
    """h_k, status and outputs after k + 1 passes, for k < passes.

    A particle still unconverged after k + 1 passes reports the h of its last evaluation,
    so solves stopped after 1, 2, ... passes expose the whole sequence of evaluated h.
    """
    runs = [oracle.solve(pos, mass, h0, targets=targets, max_iter=k + 1, **kw) for k in range(passes)]
    return runs, np.array([r["h"] for r in runs]), np.array([r["status"] for r in runs])


@pytest.mark.parametrize("case", ["uniform_scattered_starts", "clustered_common_start", "tight_clumps"])
def test_update_rule_along_trajectories(case):
    # Every step of the h iteration, checked against what the update rule fixes:
    #  - h moves towards the band (up when N_w < Nngb, down when N_w > Nngb);
    #  - it stays strictly inside the bracket of all earlier evaluations;
    #  - it is the Newton point h - (N_w - Nngb)/N_w' when that lies inside the bracket and
    #    within [h/2, 2h], otherwise the bracket midpoint, or h * 2^(1/3) (only a lower
    #    bound) or h / 2^(1/3) (only an upper bound).
    # N_w and N_w' at each evaluated h come from the fixed-h evaluation, which is pinned by
    # brute force and by finite differences above.  Each kind of step must occur.
    nngb, tol = 64.0, 0.5
    if case == "uniform_scattered_starts":
        wl = inputs.make("c1")
        tg = np.arange(0, wl.n, 17)
        h0 = wl.h0[tg] * np.random.default_rng(5).choice([0.2, 0.45, 1.0, 2.2, 4.0], size=tg.size)
        pos, mass = wl.pos, wl.mass
    elif case == "clustered_common_start":
        wl = inputs.make("c2", n=16384)
        tg = np.random.default_rng(6).choice(wl.n, size=240, replace=False)
        h0 = wl.h0[tg]
        pos, mass = wl.pos, wl.mass
    else:
        # 64 clumps of 8 (spread 2e-3) on a lattice of spacing 1/4: from h0 = 0.1 every
        # target sees N_w ~ 85 > Nngb with N_w' nearly zero, so Newton is refused and h
        # shrinks until the clump's own profile brackets the root
        g = np.arange(4) * 0.25 + 0.125
        c = np.stack([a.ravel() for a in np.meshgrid(g, g, g, indexing="ij")])
        pos = np.mod(np.repeat(c, 8, axis=1) + np.random.default_rng(7).normal(0, 2e-3, (3, 512)), 1.0)
        mass = np.full(512, 1.0 / 512)
        tg = np.arange(0, 512, 3)
        h0 = np.full(tg.size, 0.1)
    P = 14
    runs, hs, st = _trajectory(pos, mass, h0, tg, P, nngb=nngb, tol=tol)
    ev = [oracle.evaluate(pos, mass, hs[k], targets=tg) for k in range(P)]
    kinds = {"newton": 0, "midpoint": 0, "grow": 0, "shrink": 0}
    pairs = 0
    for k in range(P):
        # the outputs of an unconverged particle describe its last evaluation
        live = st[k] == oracle.STATUS_NOT_CONVERGED
        np.testing.assert_array_equal(runs[k]["rho"][live], ev[k]["rho"][live])
        np.testing.assert_array_equal(runs[k]["nw"][live], ev[k]["nw"][live])
        np.testing.assert_array_equal(runs[k]["count"][live], ev[k]["count"][live])
        # pair_evals sums the neighbour counts of every evaluation made
        evaluated = np.ones(tg.size, bool) if k == 0 else st[k - 1] == oracle.STATUS_NOT_CONVERGED
        pairs += int(ev[k]["count"][evaluated].sum())
        assert runs[k]["stats"]["pair_evals"] == pairs
        n_eval = int(evaluated.sum())
        if n_eval:
            assert runs[k]["stats"]["passes"] == k + 1
            assert runs[k]["stats"]["todo_per_pass"][k] == n_eval
        else:
            assert runs[k]["stats"]["passes"] <= k
        if k == P - 1:
            break
        for p in np.nonzero(live)[0]:
            h, nw, dnw = hs[k][p], ev[k]["nw"][p], ev[k]["dnw"][p]
            assert abs(nw - nngb) > tol
            below = [hs[j][p] for j in range(k + 1) if ev[j]["nw"][p] < nngb]
            above = [hs[j][p] for j in range(k + 1) if ev[j]["nw"][p] >= nngb]
            lo = max(below) if below else 0.0
            hi = min(above) if above else math.inf
            hn = hs[k + 1][p]
            assert (hn > h) == (nw < nngb)
            assert lo < hn < hi
            newton = h - (nw - nngb) / dnw if dnw > 0 else None
            if newton is not None and lo < newton < hi and 0.5 * h <= newton <= 2.0 * h:
                assert hn == newton
                kinds["newton"] += 1
            elif below and above:
                assert hn == 0.5 * (lo + hi)
                kinds["midpoint"] += 1
            elif below:
                assert hn == h * GROWTH
                kinds["grow"] += 1
            else:
                assert hn == h / GROWTH
                kinds["shrink"] += 1
    want = {"uniform_scattered_starts": ("newton", "grow"), "clustered_common_start": ("newton",),
            "tight_clumps": ("newton", "shrink")}[case]
    for kind in want:
        assert kinds[kind] > 0, kinds


@pytest.mark.parametrize("h,nw,dnw,lo,hi,expect,bracket", [
    # Newton accepted: 1 + (64 - 60)/40
    (1.0, 60.0, 40.0, 0.0, math.inf, 1.1, (1.0, math.inf)),
    # the Newton point 2.0 lies beyond the upper bound 1.5: midpoint of [1, 1.5]
    (1.0, 60.0, 4.0, 0.0, 1.5, 1.25, (1.0, 1.5)),
    # Newton point equal to the upper bound: the bracket is open, so the midpoint
    (1.0, 62.0, 4.0, 0.0, 1.5, 1.25, (1.0, 1.5)),
    # Newton point exactly 2h or exactly h/2: accepted (closed step limits)
    (1.0, 62.0, 2.0, 0.0, math.inf, 2.0, (1.0, math.inf)),
    (1.0, 66.0, 4.0, 0.0, math.inf, 0.5, (0.0, 1.0)),
    # beyond 2h with only a lower bound: grow by 2^(1/3)
    (1.0, 10.0, 1.0, 0.0, math.inf, GROWTH, (1.0, math.inf)),
    # below h/2 with only an upper bound: shrink by 2^(1/3)
    (1.0, 100.0, 10.0, 0.0, math.inf, 1.0 / GROWTH, (0.0, 1.0)),
    # no slope (no neighbour but the particle itself): midpoint when both bounds are set
    (0.8, 32.0 / 3.0, 0.0, 0.0, 1.0, 0.9, (0.8, 1.0)),
    (0.8, 32.0 / 3.0, 0.0, 0.0, math.inf, 0.8 * GROWTH, (0.8, math.inf)),
    # the Newton point falls below the lower bound: midpoint
    (1.2, 70.0, 20.0, 1.0, math.inf, 1.1, (1.0, 1.2)),
])
def test_h_update_branches(h, nw, dnw, lo, hi, expect, bracket):
    # Each branch of the update rule on inputs whose next h follows from the rule's
    # statement by hand; the solve applies this same step to every unconverged particle.
    hn, lo2, hi2 = oracle.h_update(h, nw, dnw, 64.0, lo, hi)
    assert hn == pytest.approx(expect, rel=1e-15)
    assert (lo2, hi2) == bracket


def test_newton_steps_converge_quadratically_at_the_closed_form_rate():
    # Two particles a distance r apart and Nngb = 16: N_w(h) = (32/3)(1 + w(r/h)) on the inner
    # piece of w, so F(h) = N_w(h) - 16 is a cubic in r/h with a simple root h*.  Newton's
    # method gives e_{k+1} = F''(h*) / (2 F'(h*)) e_k^2 + O(e_k^3); the ratio is computed here
    # symbolically from the kernel polynomial, not from the oracle.
    sympy = pytest.importorskip("sympy")
    r_sep = 0.05
    hh, q = sympy.symbols("h q", positive=True)
    w_inner = 1 - 6 * q**2 + 6 * q**3
    F = sympy.Rational(32, 3) * (1 + w_inner.subs(q, r_sep / hh)) - 16
    q_star = [x for x in sympy.Poly(6 * q**3 - 6 * q**2 + sympy.Rational(1, 2), q).nroots(n=30)
              if x.is_real and 0 < x <= sympy.Rational(1, 2)]
    assert len(q_star) == 1
    h_star = float(r_sep / q_star[0])
    c = float((sympy.diff(F, hh, 2) / (2 * sympy.diff(F, hh))).subs(hh, r_sep / q_star[0])) * h_star
    pos = np.array([[0.4, 0.4 + r_sep], [0.5, 0.5], [0.5, 0.5]])
    for f in (1.05, 0.97, 1.02):
        _, hs, st = _trajectory(pos, np.array([1.0, 1.0]), np.array([f * h_star]), np.array([0]), 7,
                                box=(0, 0, 0), periodic=False, nngb=16.0, tol=1e-13)
        assert st[5][0] == oracle.STATUS_CONVERGED  # converged within six evaluations
        e = (hs[:, 0] - h_star) / h_star
        ratios = [e[k + 1] / e[k] ** 2 for k in range(4) if 1e-7 < abs(e[k]) < 0.06]
        assert len(ratios) >= 2
        for rt in ratios:
            assert rt == pytest.approx(c, rel=0.12)


def test_band_edges_are_inclusive():
    # One isolated particle (open boundaries): N_w = 32/3 exactly at every h.  With the band
    # edge exactly on it the particle converges at once; a hair inside, it never does.
    pos = np.array([[0.5], [0.5], [0.5]])
    nw = 32.0 / 3.0
    for nngb in (10.0, 11.0):
        tol = abs(nw - nngb)  # exact (Sterbenz)
        kw = dict(box=(0, 0, 0), periodic=False, nngb=nngb, max_iter=5)
        r = oracle.solve(pos, np.array([1.0]), np.array([0.1]), tol=tol, **kw)
        assert r["status"][0] == oracle.STATUS_CONVERGED and r["stats"]["passes"] == 1
        assert r["h"][0] == 0.1
        r = oracle.solve(pos, np.array([1.0]), np.array([0.1]), tol=np.nextafter(tol, 0.0), **kw)
        assert r["status"][0] == oracle.STATUS_NOT_CONVERGED and r["stats"]["passes"] == 5


def test_a_proposal_of_half_the_box_stops_the_particle():
    # h must stay below half the periodic box: a proposed h equal to L/2 is refused before it
    # is evaluated.  h0 is the double whose 2^(1/3) growth step lands exactly on 0.5.
    h0 = 0.39685026299204984
    assert h0 * GROWTH == 0.5
    r = oracle.solve(np.array([[0.2], [0.2], [0.2]]), np.array([1.0]), np.array([h0]))
    assert r["status"][0] == oracle.STATUS_EXCEEDS_BOX
    assert r["stats"]["passes"] == 1
    assert r["h"][0] == h0
    just_below = np.nextafter(h0, 0.0)
    assert just_below * GROWTH < 0.5
    r = oracle.solve(np.array([[0.2], [0.2], [0.2]]), np.array([1.0]), np.array([just_below]))
    assert r["stats"]["passes"] == 2 and r["h"][0] == just_below * GROWTH


def test_batch_equals_groups_solved_alone():
    wl = inputs.plummer_groups(n_groups=12, nmin=32, nmax=600, seed=21)
    r = oracle.batch_solve(wl.offsets, wl.pos, wl.mass, wl.h0, wl.nngb, wl.tol)
    passes, pairs, todo = 0, 0, np.zeros(64, dtype=np.int64)
    for g in range(wl.n_groups):
        s, e = wl.offsets[g], wl.offsets[g + 1]
        a = oracle.solve(wl.pos[:, s:e], wl.mass[s:e], wl.h0[s:e], box=(0, 0, 0), periodic=False,
                         nngb=wl.nngb[g], tol=wl.tol[g])
        np.testing.assert_array_equal(a["h"], r["h"][s:e])
        np.testing.assert_array_equal(a["rho"], r["rho"][s:e])
        passes = max(passes, a["stats"]["passes"])
        pairs += a["stats"]["pair_evals"]
        todo[: a["stats"]["passes"]] += a["stats"]["todo_per_pass"]
    assert np.all(r["status"] == 0)
    assert np.all(np.abs(r["nw"] - 32.0) <= 1.0)
    # the batch runs as long as its slowest group; the work adds up over the groups
    assert r["stats"]["passes"] == passes
    assert r["stats"]["pair_evals"] == pairs
    assert r["stats"]["todo_per_pass"] == todo[:passes].tolist()


def test_batch_group_brute_force_at_solution():
    wl = inputs.plummer_groups(n_groups=5, nmin=32, nmax=3000, seed=22)
    r = oracle.batch_solve(wl.offsets, wl.pos, wl.mass, wl.h0, wl.nngb, wl.tol)
    for g in range(wl.n_groups):
        s, e = wl.offsets[g], wl.offsets[g + 1]
        b = brute.evaluate(wl.pos[:, s:e], wl.mass[s:e], r["h"][s:e], periodic=False)
        np.testing.assert_array_equal(b["count"], r["count"][s:e])
        np.testing.assert_allclose(b["rho"], r["rho"][s:e], rtol=1e-13)


# --------------------------------------------------------------------------------------
# Wendland C6 (the paper's kernel, Sec. II-B)
# --------------------------------------------------------------------------------------

def test_wendland_c6_normalisation_and_shape():
    # int W d^3r = 1365/(64 pi) * 4 pi * int q^2 w = (1365/16) int_0^1 q^2 w(q) dq = 1
    val, _ = integrate.quad(lambda q: q * q * oracle.w_c6(q), 0.0, 1.0, epsabs=1e-15, epsrel=1e-14)
    assert abs(1365.0 / 16.0 * val - 1.0) < 1e-12
    assert oracle.w_c6(0.0) == 1.0
    for q in (1.0, 1.2, 3.0):
        assert oracle.w_c6(q) == 0.0 and oracle.mqdw_c6(q) == 0.0
    # contact of order 8 at the support edge (C6 for the radial function): w(1-e)/e^8 -> w's
    # polynomial factor at q = 1, which is 1 + 8 + 25 + 32 = 66
    for e in (1e-2, 1e-3):
        assert oracle.w_c6(1.0 - e) / e**8 == pytest.approx(66.0, rel=0.2 * e / 1e-2)
    # even at the origin: no linear term
    assert abs((oracle.w_c6(1e-6) - 1.0) / 1e-6) < 1e-4


def test_wendland_c6_mqdw_is_minus_q_derivative():
    for q in np.linspace(0.02, 0.98, 49):
        d1, _ = _derivs(oracle.w_c6, q, 1e-6)
        assert oracle.mqdw_c6(q) == pytest.approx(-q * d1, rel=1e-6, abs=1e-9)


def test_wendland_c6_matches_brute_force_and_finite_difference():
    wl = inputs.uniform_box(n=3000, seed=17, nngb=295.0)
    rng = np.random.default_rng(2)
    h = wl.h0 * rng.uniform(0.8, 1.2, size=wl.n)
    o = oracle.evaluate(wl.pos, wl.mass, h, kernel="wendland_c6")
    b = brute.evaluate(wl.pos, wl.mass, h, kernel="wendland_c6")
    np.testing.assert_array_equal(o["count"], b["count"])
    np.testing.assert_allclose(o["rho"], b["rho"], rtol=1e-13)
    np.testing.assert_allclose(o["nw"], b["nw"], rtol=1e-13)
    tg = np.arange(0, wl.n, 97)
    eps = 1e-7
    up = oracle.evaluate(wl.pos, wl.mass, h[tg] * (1 + eps), targets=tg, kernel="wendland_c6")
    dn = oracle.evaluate(wl.pos, wl.mass, h[tg] * (1 - eps), targets=tg, kernel="wendland_c6")
    fd = (up["nw"] - dn["nw"]) / (2 * eps * h[tg])
    np.testing.assert_allclose(o["dnw"][tg], fd, rtol=2e-5)
    # for a uniform Poisson field the neighbours other than the particle itself contribute
    # n m int W = the mean density on average; the self term m W(0) comes on top
    self_term = wl.mass * 1365.0 / (64.0 * math.pi * h**3)
    assert abs(np.mean(o["rho"] - self_term) - 1.0) < 0.01
    assert np.median(o["rho"]) > 1.05  # the self term is ~10 % at 295 neighbours


def test_wendland_c6_solve_converges_in_band():
    wl = inputs.uniform_box(n=4096, seed=18, nngb=295.0)
    r = oracle.solve(wl.pos, wl.mass, wl.h0, nngb=295.0, tol=5.0, kernel="wendland_c6")
    assert np.all(r["status"] == 0)
    assert np.all(np.abs(r["nw"] - 295.0) <= 5.0)


# ---- k-nearest-neighbour smoothing length (Sec. IV-D) --------------------------------------

def _lattice(side):
    """Simple cubic lattice of side^3 particles with spacing a = 1/side in the unit periodic box
    (positions are exact binary fractions, so every squared distance is exact)."""
    a = 1.0 / side
    g = np.arange(side) * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()])
    return pos, np.full(side**3, 1.0 / side**3), a


@pytest.mark.parametrize("kernel", ["m4", "wendland_c6"])
def test_knn_lattice_shells_closed_form(kernel):
    # shells of the simple cubic lattice: 1 (self), 6 at a, 12 at sqrt(2) a, 8 at sqrt(3) a,
    # 6 at 2a.  The K-th nearest distance is the shell radius holding the K-th particle, and
    # the density sums the shells strictly inside it (the K-th shell sits at q = 1, w = 0).
    pos, m, a = _lattice(8)
    wfun = oracle.w if kernel == "m4" else oracle.w_c6
    sigma = 8.0 / math.pi if kernel == "m4" else 1365.0 / (64.0 * math.pi)
    shells = [(0.0, 1), (a, 6), (math.sqrt(2) * a, 12), (math.sqrt(3) * a, 8), (2 * a, 6)]
    for k, hk, inner in ((2, a, 1), (7, a, 1), (8, math.sqrt(2) * a, 2), (19, math.sqrt(2) * a, 2),
                         (20, math.sqrt(3) * a, 3), (27, math.sqrt(3) * a, 3), (33, 2 * a, 4)):
        r = oracle.knn(pos, m, k, targets=np.arange(0, 512, 37), kernel=kernel)
        assert np.all(r["status"] == 0)
        np.testing.assert_allclose(r["h"], hk, rtol=2e-16)
        rho = m[0] * sigma / hk**3 * sum(c * wfun(rad / hk) for rad, c in shells[:inner])
        np.testing.assert_allclose(r["rho"], rho, rtol=1e-14)
        below = sum(c for _, c in shells[:inner])
        # the K-th shell itself is counted only if fl(h)^2 rounds above its squared radius
        assert np.all((r["count"] == below) | (r["count"] == below + shells[inner][1]))


@pytest.mark.parametrize("periodic", [True, False])
def test_knn_matches_kdtree_kth_distance(periodic):
    spatial = pytest.importorskip("scipy.spatial")
    wl = inputs.make("c1", n=3000)
    pos = wl.pos
    tg = np.arange(0, wl.n, 7)
    for k in (2, 33, 64, 295):
        r = oracle.knn(pos, wl.mass, k, periodic=periodic, targets=tg)
        tree = spatial.cKDTree(pos.T, boxsize=1.0 if periodic else None)
        d, _ = tree.query(pos.T[tg], k=k)
        np.testing.assert_allclose(r["h"], d[:, -1], rtol=1e-14)


def test_knn_bracket_and_density_at_h():
    # the K-th distance brackets the K nearest: fewer than K particles strictly closer, at
    # least K at or within it; and the density is the fixed-h evaluation at that h
    wl = inputs.make("c2", n=4096)
    tg = np.arange(0, wl.n, 13)
    k = 64
    r = oracle.knn(wl.pos, wl.mass, k, targets=tg)
    d = wl.pos[:, tg, None] - wl.pos[:, None, :]
    d -= np.round(d)
    dist = np.sqrt((d**2).sum(0))
    assert np.all((dist < r["h"][:, None] * (1 - 1e-12)).sum(1) < k)
    assert np.all((dist <= r["h"][:, None] * (1 + 1e-12)).sum(1) >= k)
    e = oracle.evaluate(wl.pos, wl.mass, r["h"], targets=tg)
    np.testing.assert_array_equal(r["rho"], e["rho"])
    np.testing.assert_array_equal(r["count"], e["count"])
    b = oracle.knn(wl.pos, wl.mass, k, targets=tg, mode="brute")
    np.testing.assert_array_equal(b["h"], r["h"])
    np.testing.assert_allclose(b["rho"], r["rho"], rtol=1e-13)


def test_knn_exceeds_box_and_argument_range():
    pos, m, a = _lattice(3)  # 27 particles, spacing 1/3: the 27th-nearest is at sqrt(3)/3 > 1/2
    r = oracle.knn(pos, m, 27, targets=np.arange(3))
    assert np.all(r["status"] == 2)
    r = oracle.knn(pos, m, 7, targets=np.arange(3))  # 1/3 < 1/2
    assert np.all(r["status"] == 0)
    for k in (1, 28):
        with pytest.raises(ValueError):
            oracle.knn(pos, m, k)
    # a K-th distance of exactly half the box is already beyond the periodic limit
    two = np.array([[0.0, 0.5], [0.0, 0.0], [0.0, 0.0]])
    r = oracle.knn(two, np.ones(2), 2)
    assert np.all(r["h"] == 0.5) and np.all(r["status"] == 2)
    two[0, 1] = 0.375
    r = oracle.knn(two, np.ones(2), 2)
    assert np.all(r["h"] == 0.375) and np.all(r["status"] == 0)
