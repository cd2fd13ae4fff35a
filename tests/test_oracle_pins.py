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


def test_batch_equals_groups_solved_alone():
    wl = inputs.plummer_groups(n_groups=12, nmin=32, nmax=600, seed=21)
    r = oracle.batch_solve(wl.offsets, wl.pos, wl.mass, wl.h0, wl.nngb, wl.tol)
    for g in range(wl.n_groups):
        s, e = wl.offsets[g], wl.offsets[g + 1]
        a = oracle.solve(wl.pos[:, s:e], wl.mass[s:e], wl.h0[s:e], box=(0, 0, 0), periodic=False,
                         nngb=wl.nngb[g], tol=wl.tol[g])
        np.testing.assert_array_equal(a["h"], r["h"][s:e])
        np.testing.assert_array_equal(a["rho"], r["rho"][s:e])
    assert np.all(r["status"] == 0)
    assert np.all(np.abs(r["nw"] - 32.0) <= 1.0)


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
