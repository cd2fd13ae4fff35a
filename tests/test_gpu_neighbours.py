"""Neighbour sets, not only counts: the GPU's in-h decisions pair by pair.

sph_neighbours_sampled runs one fixed-h density pass exactly as sph_density_eval does and
records, for sampled targets, the particles that pass the distance test r_ij < h_i, i.e. the
neighbour list (ngblist) that Listing 1 loops over and Eq. (1) sums over.  Each list is
compared with an FP64 brute-force search in NumPy (minimum image):
  - FP64 mode forms every distance as the FP64 formulae are written, so the sets must be equal;
  - FP32 mode tests FP32 offsets from 32-bit fixed-point coordinates, so a pair may be decided
    differently only when its FP64 distance lies within 1e-6 h of the boundary (the rounding
    bound derived for that test); every other pair must agree.
The pass's own counts and densities must also equal those of sph_density_eval on the same
inputs (the export changes nothing but the recording).
"""
import numpy as np
import pytest

from paper_1612_06090_gb300 import inputs
from tests import brute

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1612_06090_gb300 import binding as B  # noqa: E402

FP64, FP32 = B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN
DEV = torch.device("cuda:0")
BAND = 1e-6  # FP32: pairs within BAND * h of the boundary may be decided either way


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def gpu_neighbours(pos, mass, h, sample, precision, max_nbr=None, box=(1.0, 1.0, 1.0), **kw):
    s = B.Solver(len(mass), precision=precision, box=box, **kw)
    s.sort(T(pos), T(mass))
    if max_nbr is None:
        # the counts are complete even when the rows are cut: size the rows from a first call
        first = s.neighbours(T(h), T(sample, torch.int64), 1)
        max_nbr = int(first["nbr_count"].max().item())
    r = s.neighbours(T(h), T(sample, torch.int64), max_nbr)
    ev = s.evaluate(T(h))
    torch.cuda.synchronize()
    nbr = r["nbr"].cpu().numpy()
    cnt = r["nbr_count"].cpu().numpy()
    assert np.all(cnt <= max_nbr), "max_nbr too small for this case"
    lists = [np.sort(nbr[k, :cnt[k]]) for k in range(len(sample))]
    # the export pass is the evaluation pass: same counts and densities
    np.testing.assert_array_equal(r["count"].cpu().numpy(), ev["count"].cpu().numpy())
    np.testing.assert_array_equal(r["rho"].cpu().numpy(), ev["rho"].cpu().numpy())
    np.testing.assert_array_equal(cnt, ev["count"].cpu().numpy()[sample])
    s.close()
    return lists


def compare_sets(gpu_lists, pos, h, sample, box=(1.0, 1.0, 1.0), exact=True):
    """Returns (pairs differing, largest |r - h| / h among them)."""
    inside, near = brute.neighbours(pos, h[sample], sample, box=box, band=0.0 if exact else 4 * BAND)
    n_diff, worst = 0, 0.0
    for k, i in enumerate(sample):
        g, b = gpu_lists[k], inside[k]
        assert np.unique(g).size == g.size, f"target {i}: a neighbour recorded twice"
        if exact:
            np.testing.assert_array_equal(g, b, err_msg=f"target {i}")
            continue
        diff = np.setxor1d(g, b)
        for j in diff:
            r = near[k].get(int(j))
            assert r is not None, f"target {i}, particle {j}: decided differently far from the boundary"
            rel = abs(r - h[i]) / h[i]
            worst = max(worst, rel)
            assert rel <= BAND, (i, int(j), rel)
        n_diff += diff.size
    return n_diff, worst


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("scale", [0.55, 1.0, 1.9])
def test_neighbour_sets_uniform_config1(precision, scale):
    wl = inputs.make("c1")
    rng = np.random.default_rng(17)
    h = wl.h0 * scale * rng.uniform(0.9, 1.1, size=wl.n)
    sample = np.arange(wl.n)
    g = gpu_neighbours(wl.pos, wl.mass, h, sample, precision)
    n_diff, worst = compare_sets(g, wl.pos, h, sample, exact=precision == FP64)
    print(f"c1 scale {scale}: {n_diff} pairs decided differently, worst |r-h|/h {worst:.2e}")


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_neighbour_sets_adversarial_positions(precision):
    # particles on the cell faces of a 64^3 grid, at the box corners and at the periodic seam,
    # with h on exact grid distances (plus 1e-9) so that many pairs sit right at r = h
    rng = np.random.default_rng(5)
    k = rng.integers(0, 64, size=(3, 3000))
    pos = k / 64.0
    pos[:, :6] = np.array([[0, 0, 0], [1 - 2**-30, 0, 0], [0, 1 - 2**-30, 0],
                           [0, 0, 1 - 2**-30], [0.5, 0.5, 0.5], [1 - 2**-40, 1 - 2**-40, 0.0]]).T
    mass = rng.uniform(0.5, 1.5, size=3000)
    h = np.full(3000, 0.1)
    h[::3] = 1.0 / 16.0 + 1e-9
    h[1::3] = 3.0 / 64.0 + 1e-9
    sample = np.arange(3000)
    g = gpu_neighbours(pos, mass, h, sample, precision)
    compare_sets(g, pos, h, sample, exact=precision == FP64)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_neighbour_sets_wendland_c6(precision):
    wl = inputs.uniform_box(n=20000, seed=61, nngb=295.0)
    rng = np.random.default_rng(9)
    h = wl.h0 * rng.uniform(0.7, 1.3, size=wl.n)
    sample = np.sort(rng.choice(wl.n, size=600, replace=False))
    g = gpu_neighbours(wl.pos, wl.mass, h, sample, precision,
                       kernel=B.SPH_KERNEL_WENDLAND_C6, nngb=295.0, tol=5.0)
    compare_sets(g, wl.pos, h, sample, exact=precision == FP64)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_neighbour_sets_anisotropic_box(precision):
    rng = np.random.default_rng(12)
    box = (1.0, 2.0, 0.5)
    n = 4000
    pos = np.stack([rng.uniform(0, box[d], n) for d in range(3)])
    mass = rng.uniform(0.5, 2.0, n)
    h = np.full(n, inputs.mean_density_h(64.0, n / (box[0] * box[1] * box[2]))) * rng.uniform(0.6, 1.5, n)
    sample = np.arange(n)
    g = gpu_neighbours(pos, mass, h, sample, precision, box=box)
    compare_sets(g, pos, h, sample, box=box, exact=precision == FP64)


@pytest.mark.parametrize("spread", ["uniform_h0", "lognormal"])
@pytest.mark.parametrize("precision", [FP32, FP64])
def test_neighbour_sets_config2_sampled(precision, spread):
    """The 1,048,576-particle Plummer-cluster set.  uniform_h0: every h = h0, the cold start's
    first pass (the branch-free FP32 loop; thousands of neighbours in the sphere cores);
    lognormal: h spread over a factor of ~10 around h0, so work items hold targets of very
    different h (the later passes' situation)."""
    wl = inputs.make("c2")
    rng = np.random.default_rng(2025)
    if spread == "uniform_h0":
        h = wl.h0.copy()
    else:
        h = wl.h0 * np.exp(rng.normal(0.0, 0.6, size=wl.n))
        h = np.minimum(h, 0.2)
    sample = np.sort(rng.choice(wl.n, size=300, replace=False))
    g = gpu_neighbours(wl.pos, wl.mass, h, sample, precision)
    n_diff, worst = compare_sets(g, wl.pos, h, sample, exact=precision == FP64)
    print(f"c2 {spread}: {n_diff} pairs decided differently, worst |r-h|/h {worst:.2e}")


def test_neighbour_export_argument_errors():
    wl = inputs.make("c1")
    s = B.Solver(wl.n, precision=FP32)
    h = T(wl.h0)
    nbr = torch.empty((4, 8), dtype=torch.int32, device=DEV)
    cnt = torch.empty(4, dtype=torch.int32, device=DEV)
    rho = torch.empty(wl.n, dtype=torch.float64, device=DEV)
    c = torch.empty(wl.n, dtype=torch.int32, device=DEV)
    smp = T([0, 1, 2, 3], torch.int64)
    call = lambda sm, ns=4, mx=8: B.sph_neighbours_sampled(  # noqa: E731
        s.ctx, h.data_ptr(), ns, sm.data_ptr(), mx, nbr.data_ptr(), cnt.data_ptr(), rho.data_ptr(), c.data_ptr())
    assert call(smp) == B.SPH_ERR_NOT_SORTED
    s.sort(T(wl.pos), T(wl.mass))
    assert call(smp, ns=0) == B.SPH_ERR_INVALID_ARG
    assert call(smp, mx=0) == B.SPH_ERR_INVALID_ARG
    assert call(T([0, 1, 1, 3], torch.int64)) == B.SPH_ERR_INVALID_ARG  # repeated
    assert call(T([0, 1, wl.n, 3], torch.int64)) == B.SPH_ERR_INVALID_ARG  # out of range
    assert call(T([0, -1, 2, 3], torch.int64)) == B.SPH_ERR_INVALID_ARG
    assert call(smp) == B.SPH_OK
    # a row with more neighbours than max_nbr: the count is complete, only max_nbr are written
    torch.cuda.synchronize()
    assert np.all(cnt.cpu().numpy() == c.cpu().numpy()[:4])
    s.close()


@pytest.mark.parametrize("precision", [FP32, FP64])
def test_neighbour_sets_lognormal_16M_at_converged_h(precision):
    """Full size: the 16.7M-particle log-normal field at its FP32-converged h (densities over
    orders of magnitude, the late passes' sparse targets included), sampled targets against the
    brute-force sets over every particle."""
    wl = inputs.make("c3")
    s = B.Solver(wl.n, precision=FP32, box=wl.box, nngb=wl.nngb, tol=wl.tol, use_graph=True)
    s.sort(T(wl.pos), T(wl.mass))
    r = s.solve(T(wl.h0))
    assert r["status"] == B.SPH_OK
    h = r["h"].cpu().numpy()
    s.close()
    rng = np.random.default_rng(163)
    sample = np.sort(rng.choice(wl.n, size=24, replace=False))
    g = gpu_neighbours(wl.pos, wl.mass, h, sample, precision, box=wl.box)
    compare_sets(g, wl.pos, h, sample, box=wl.box, exact=precision == FP64)
