"""Pins of the oracle's velocity-field pair sums (oracle.interact), the further pair
computations over the neighbour sets of Eq. (1) (Listing 1, the second interaction phase).

What fixes them without retyping the oracle's formulas:
- two particles: closed forms, with w'(q) from sympy's derivative of the shape polynomials;
- a uniform velocity field: the mean is that velocity, dispersion, divergence and curl vanish;
- a Galilean boost changes the mean by the boost and nothing else;
- a linear field v = A r on a cubic lattice: by the lattice's symmetry the mean is A r_i, the
  divergence is K tr(A), the curl of a rotation with angular velocity w is 2 K w with the same
  K, and the dispersion is |A|_F^2 times one constant; integration by parts gives K -> 1 and
  the constant -> (1/3) of the kernel's second moment as the neighbours grow dense;
- an independent NumPy brute force (tests/brute.py) written in a different but equivalent form;
- rho and the neighbour count equal the density evaluation's.
"""
import math

import numpy as np
import pytest

import oracle
from tests import brute

KERNELS = ["m4", "wendland_c6"]


def _sym_shapes(kernel):
    sp = pytest.importorskip("sympy")
    q = sp.symbols("q", nonnegative=True)
    if kernel == "m4":
        pieces = [(1 - 6 * q**2 + 6 * q**3, 0.0, 0.5), (2 * (1 - q) ** 3, 0.5, 1.0)]
        sigma = 8 / math.pi
    else:
        pieces = [((1 - q) ** 8 * (1 + 8 * q + 25 * q**2 + 32 * q**3), 0.0, 1.0)]
        sigma = 1365 / (64 * math.pi)

    def w(x):
        for f, a, b in pieces:
            if a <= x <= b:
                return float(f.subs(q, x))
        return 0.0

    def dw(x):
        for f, a, b in pieces:
            if a <= x <= b:
                return float(sp.diff(f, q).subs(q, x))
        return 0.0

    return w, dw, sigma


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("qv", [0.31, 0.77])
def test_two_particles_closed_form(kernel, qv):
    w, dw, sigma = _sym_shapes(kernel)
    h = 0.2
    rvec = np.array([0.6, -0.48, 0.64])  # |rvec| = 1
    pi_ = np.array([0.3, 0.4, 0.5])
    pj = pi_ + qv * h * rvec
    pos = np.stack([pi_, pj], axis=1)
    mi, mj = 1.5, 0.7
    vi, vj = np.array([0.1, -0.2, 0.3]), np.array([-0.4, 0.25, 0.9])
    vel = np.stack([vi, vj], axis=1)
    o = oracle.interact(pos, np.array([mi, mj]), vel, h, periodic=False, targets=[0], kernel=kernel)
    a, b = mi * w(0.0), mj * w(qv)
    rho = sigma / h**3 * (a + b)
    vbar = (a * vi + b * vj) / (a + b)
    sig2 = a * b / (a + b) ** 2 * np.dot(vj - vi, vj - vi)
    grad = sigma / h**4 * dw(qv) * (pi_ - pj) / (qv * h)  # dW/dr along r_i - r_j
    div = mj * np.dot(vj - vi, grad) / rho
    curl = mj * np.cross(vi - vj, grad) / rho
    assert o["count"][0] == 2
    assert o["rho"][0] == pytest.approx(rho, rel=1e-13)
    np.testing.assert_allclose(o["vmean"][:, 0], vbar, rtol=1e-13, atol=1e-15)
    assert o["sigma2"][0] == pytest.approx(sig2, rel=1e-12)
    assert o["div"][0] == pytest.approx(div, rel=1e-12)
    np.testing.assert_allclose(o["curl"][:, 0], curl, rtol=1e-12, atol=1e-12 * np.abs(curl).max())
    # the kernel falls off with r: a pair approaching each other converges (negative divergence)
    o2 = oracle.interact(pos, np.array([mi, mj]), np.stack([np.zeros(3), -rvec], axis=1), h,
                         periodic=False, targets=[0], kernel=kernel)
    assert o2["div"][0] < 0.0


def _within(a, b, tol):
    """|a - b| <= tol elementwise (tol may be one bound per target)."""
    err = np.abs(np.asarray(a) - np.asarray(b))
    assert np.all(err <= tol), float(np.max(err / np.maximum(tol, 1e-300)))


def _random_set(seed, n=1200):
    rng = np.random.default_rng(seed)
    pos = rng.random((3, n))
    m = rng.uniform(0.5, 1.5, n) / n
    vel = rng.normal(size=(3, n)) + np.array([[2.0], [0.0], [-1.0]])
    h = rng.uniform(0.08, 0.16, n)
    return pos, m, vel, h


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("periodic", [True, False])
def test_matches_numpy_brute_force(kernel, periodic):
    pos, m, vel, h = _random_set(11)
    box = (1.0, 0.8, 1.3)  # unequal sides: each periodic image uses its own length
    pos = pos * np.array(box)[:, None]
    o = oracle.interact(pos, m, vel, h, box=box, periodic=periodic, kernel=kernel)
    ob = oracle.interact(pos, m, vel, h, box=box, periodic=periodic, kernel=kernel, mode="brute")
    b = brute.interact(pos, m, vel, h, box=box, periodic=periodic, kernel=kernel)
    for ref in (ob, b):
        np.testing.assert_array_equal(o["count"], ref["count"])
        np.testing.assert_allclose(o["rho"], ref["rho"], rtol=1e-13)
        np.testing.assert_allclose(o["vmean"], ref["vmean"], rtol=0, atol=1e-13 * o["vmax"].max())
        _within(o["sigma2"], ref["sigma2"], 1e-12 * o["vscale2"] + 1e-26 * o["vmax"] ** 2)
        _within(o["div"], ref["div"], 1e-12 * o["gabs"])
        _within(o["curl"], ref["curl"], 1e-12 * o["gabs"])
    e = oracle.evaluate(pos, m, h, box=box, periodic=periodic, kernel=kernel)
    np.testing.assert_array_equal(o["count"], e["count"])
    np.testing.assert_allclose(o["rho"], e["rho"], rtol=1e-13)


@pytest.mark.parametrize("kernel", KERNELS)
def test_uniform_field_and_galilean_boost(kernel):
    pos, m, vel, h = _random_set(12, n=800)
    c = np.array([3.0, -1.25, 0.5])
    o = oracle.interact(pos, m, np.repeat(c[:, None], pos.shape[1], axis=1), h, kernel=kernel)
    np.testing.assert_allclose(o["vmean"], np.repeat(c[:, None], pos.shape[1], axis=1), rtol=1e-14)
    assert np.all(np.abs(o["sigma2"]) <= 1e-28)
    assert np.all(o["div"] == 0.0) and np.all(o["curl"] == 0.0)
    a = oracle.interact(pos, m, vel, h, kernel=kernel)
    b = oracle.interact(pos, m, vel + c[:, None], h, kernel=kernel)
    np.testing.assert_allclose(b["vmean"] - c[:, None], a["vmean"], rtol=0, atol=1e-13 * b["vmax"].max())
    _within(b["sigma2"], a["sigma2"], 1e-12 * a["vscale2"] + 1e-26 * b["vmax"] ** 2)
    _within(b["div"], a["div"], 1e-12 * a["gabs"])
    _within(b["curl"], a["curl"], 1e-12 * a["gabs"])


def _lattice(L=20):
    g = (np.arange(L) + 0.5) / L
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    return pos, np.full(pos.shape[1], 1.0 / pos.shape[1])


@pytest.mark.parametrize("kernel", KERNELS)
def test_linear_field_on_a_lattice(kernel):
    L = 20
    pos, m = _lattice(L)
    h = 5.2 / L
    # interior targets: every neighbour of theirs is on the lattice
    tg = np.flatnonzero(np.all(np.abs(pos - 0.5) <= 0.5 - h - 1e-9, axis=0))[::97][:6]
    c = np.full(3, 0.5)
    rel = pos - c[:, None]
    omega = np.array([0.3, -0.2, 0.5])
    Arot = np.array([[0.0, -omega[2], omega[1]], [omega[2], 0.0, -omega[0]], [-omega[1], omega[0], 0.0]])
    Asym = np.array([[0.4, 0.2, -0.1], [0.2, -0.1, 0.3], [-0.1, 0.3, -0.3]])  # traceless
    Aexp = 0.7 * np.eye(3)
    res = {}
    for name, A in (("rot", Arot), ("sym", Asym), ("exp", Aexp)):
        o = oracle.interact(pos, m, A @ rel, h, periodic=False, targets=tg, kernel=kernel)
        res[name] = o
        np.testing.assert_allclose(o["vmean"], (A @ rel)[:, tg], rtol=0, atol=1e-14)
    K = res["exp"]["div"] / (3 * 0.7)
    # one consistency factor for the divergence of an expansion and the curl of a rotation
    np.testing.assert_allclose(res["rot"]["curl"] / (2 * omega[:, None]), np.broadcast_to(K, (3, tg.size)),
                               rtol=1e-12)
    assert np.all(np.abs(res["rot"]["div"]) <= 1e-13)
    assert np.all(np.abs(res["sym"]["div"]) <= 1e-13)
    assert np.all(np.abs(res["sym"]["curl"]) <= 1e-13)
    assert np.all(np.abs(res["exp"]["curl"]) <= 1e-13)
    # integration by parts: -(1/3) int r dW/dr d^3r = int W d^3r = 1
    assert np.all(np.abs(K - 1.0) < 1e-3)
    # dispersion = |A|_F^2 (1/3) <r^2>_W; the continuum second moment is 3/40 h^2 (M4) and
    # 1/24 h^2 (Wendland C6) by quadrature of the shape
    from scipy.integrate import quad

    w, _, sigma = _sym_shapes(kernel)
    moment = quad(lambda x: w(x) * x**4, 0.0, 1.0, points=[0.5])[0] * sigma * 4.0 * math.pi / 3.0
    for name, A in (("rot", Arot), ("sym", Asym), ("exp", Aexp)):
        ratio = res[name]["sigma2"] / np.sum(A * A) / (h * h)
        np.testing.assert_allclose(ratio, moment, rtol=1e-3)
    np.testing.assert_allclose(res["rot"]["sigma2"] / np.sum(Arot**2), res["sym"]["sigma2"] / np.sum(Asym**2),
                               rtol=1e-12)
