"""GPU parity of the k-nearest-neighbour smoothing length (Sec. IV-D) through the C ABI.

h_i is the distance to the K-th nearest particle (the particle itself first) and rho_i the
density at that h.  FP64 forms every squared distance exactly as the oracle does and the
K-th smallest value is unique, so h agrees bit for bit, counts exactly, and rho to summation
order.  FP32 selects among FP32 squared distances of offsets quantised to box/2^32: h agrees
to 2e-6 relative (another particle can be K-th only when its distance is that close), rho
to 1e-5, and counts within the pairs the oracle finds within 1e-6 h of the boundary.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1612_06090_gb300 import inputs
from tests.parity import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1612_06090_gb300 import binding as B  # noqa: E402

FP64, FP32 = B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN
DEV = torch.device("cuda:0")


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def gpu_knn(pos, mass, k, h0, precision, box=(1.0, 1.0, 1.0), kernel=B.SPH_KERNEL_M4, max_iter=64):
    s = B.Solver(len(mass), precision=precision, box=box, kernel=kernel, max_iter=max_iter,
                 nngb=64.0 if kernel == B.SPH_KERNEL_M4 else 295.0)
    s.sort(T(pos), T(mass))
    r = s.knn(k, T(np.array(np.broadcast_to(h0, (len(mass),)))))
    torch.cuda.synchronize()
    out = {key: (v.detach().cpu().numpy() if torch.is_tensor(v) else v) for key, v in r.items()}
    s.close()
    return out


def check_fp32(g, pos, mass, tg, k, o, kernel="m4"):
    assert np.max(rel_err(g["h"][tg], o["h"])) <= 2e-6
    assert np.max(rel_err(g["rho"][tg], o["rho"])) <= 1e-5
    e = oracle.evaluate(pos, mass, g["h"][tg], targets=tg, near_rel=1e-6, kernel=kernel)
    assert np.all(np.abs(g["count"][tg].astype(np.int64) - e["count"]) <= e["near"])


@pytest.mark.parametrize("cfg,n", [("c1", 4096), ("c2", 16384)])
@pytest.mark.parametrize("k", [2, 33, 64, 295])
def test_knn_fp64_bit_exact(cfg, n, k):
    wl = inputs.make(cfg, n=n)
    rng = np.random.default_rng(k)
    # starting radii from far too small to far too large, and 0 (estimated from the local cell
    # density): only the number of passes changes
    h0 = wl.h0 * rng.choice([0.0, 0.3, 1.0, 3.0], size=wl.n)
    g = gpu_knn(wl.pos, wl.mass, k, h0, FP64)
    assert g["status"] == B.SPH_OK
    assert g["stats"]["unconverged"] == 0
    tg = np.arange(0, wl.n, 3)
    o = oracle.knn(wl.pos, wl.mass, k, targets=tg)
    np.testing.assert_array_equal(g["h"][tg], o["h"])
    np.testing.assert_array_equal(g["count"][tg], o["count"])
    assert np.max(rel_err(g["rho"][tg], o["rho"])) <= 1e-12


@pytest.mark.parametrize("cfg,n", [("c1", 4096), ("c2", 16384)])
@pytest.mark.parametrize("k", [2, 64, 295, 512])
def test_knn_fp32_against_oracle(cfg, n, k):
    wl = inputs.make(cfg, n=n)
    g = gpu_knn(wl.pos, wl.mass, k, wl.h0, FP32)
    assert g["status"] == B.SPH_OK
    tg = np.arange(0, wl.n, 5)
    o = oracle.knn(wl.pos, wl.mass, k, targets=tg)
    check_fp32(g, wl.pos, wl.mass, tg, k, o)


def test_knn_wendland_c6_fp32_and_fp64():
    wl = inputs.make("c2", n=16384)
    tg = np.arange(0, wl.n, 7)
    o = oracle.knn(wl.pos, wl.mass, 295, targets=tg, kernel="wendland_c6")
    g = gpu_knn(wl.pos, wl.mass, 295, wl.h0 * 1.7, FP64, kernel=B.SPH_KERNEL_WENDLAND_C6)
    np.testing.assert_array_equal(g["h"][tg], o["h"])
    assert np.max(rel_err(g["rho"][tg], o["rho"])) <= 1e-12
    g = gpu_knn(wl.pos, wl.mass, 295, wl.h0 * 1.7, FP32, kernel=B.SPH_KERNEL_WENDLAND_C6)
    check_fp32(g, wl.pos, wl.mass, tg, 295, o, kernel="wendland_c6")


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_knn_lattice_ties(precision):
    # 8^3 simple cubic lattice: whole shells of equal distances (6, 12, 8, 6 particles); the
    # K-th distance is the shell radius, whichever particle of the shell is called K-th
    side = 8
    a = 1.0 / side
    gr = np.arange(side) * a
    x, y, z = np.meshgrid(gr, gr, gr, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()])
    m = np.full(side**3, 1.0 / side**3)
    for k, hk in ((7, a), (19, math.sqrt(2) * a), (27, math.sqrt(3) * a), (33, 2 * a)):
        g = gpu_knn(pos, m, k, 1.1 * a, precision)
        assert g["status"] == B.SPH_OK
        np.testing.assert_allclose(g["h"], hk, rtol=2e-16)
        o = oracle.knn(pos, m, k, targets=np.arange(0, side**3, 17))
        np.testing.assert_allclose(g["rho"][::17], o["rho"], rtol=1e-12 if precision == FP64 else 1e-6)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_knn_exceeds_box(precision):
    wl = inputs.make("c1", n=64)
    k = 32  # the 32nd of 64: beyond half the box for 19 targets, within it for the others
    g = gpu_knn(wl.pos, wl.mass, k, 0.2, precision)  # a legal start: below half the box
    o = oracle.knn(wl.pos, wl.mass, k)
    n_ex = int(np.sum(o["status"] == 2))
    assert 0 < n_ex < wl.n
    assert g["status"] == B.SPH_ERR_H_EXCEEDS_BOX
    assert g["stats"]["exceeded"] == n_ex
    ok = o["status"] == 0
    if precision == FP64:
        np.testing.assert_array_equal(g["h"][ok], o["h"][ok])
    else:
        assert np.max(rel_err(g["h"][ok], o["h"][ok])) <= 2e-6
    # every reported h is a legal radius
    assert np.all(g["h"] < 0.5)


def test_knn_pass_limit_reports_not_converged():
    wl = inputs.make("c1", n=4096)
    g = gpu_knn(wl.pos, wl.mass, 64, wl.h0 * 1e-3, FP32, max_iter=1)
    assert g["status"] == B.SPH_ERR_NOT_CONVERGED
    assert g["stats"]["unconverged"] > 0
    assert g["stats"]["passes"] == 1


def test_knn_argument_errors():
    wl = inputs.make("c1", n=256)
    s = B.Solver(wl.n, precision=FP32)
    h = T(wl.h0)
    rho = torch.empty_like(h)
    cnt = torch.empty(wl.n, dtype=torch.int32, device=DEV)
    assert B.sph_knn_solve(s.ctx, 64, h.data_ptr(), rho.data_ptr(), cnt.data_ptr()) == B.SPH_ERR_NOT_SORTED
    s.sort(T(wl.pos), T(wl.mass))
    for k in (1, 0, B.SPH_KNN_MAX_K + 1, wl.n + 1):
        assert B.sph_knn_solve(s.ctx, k, h.data_ptr(), rho.data_ptr(), cnt.data_ptr()) == B.SPH_ERR_INVALID_ARG
    assert B.sph_knn_solve(s.ctx, 64, 0, rho.data_ptr(), cnt.data_ptr()) == B.SPH_ERR_INVALID_ARG
    for v in (float("nan"), float("inf"), 0.5):  # not a radius, or not below half the box
        bad = torch.full_like(h, v)
        assert B.sph_knn_solve(s.ctx, 64, bad.data_ptr(), rho.data_ptr(), cnt.data_ptr()) == B.SPH_ERR_DEVICE_STATUS
    s.close()


def test_knn_estimated_radius_fp32():
    # every starting radius estimated from the cell table (the bench's start)
    wl = inputs.make("c2", n=16384)
    g = gpu_knn(wl.pos, wl.mass, 295, 0.0, FP32)
    assert g["status"] == B.SPH_OK
    tg = np.arange(0, wl.n, 5)
    check_fp32(g, wl.pos, wl.mass, tg, 295, oracle.knn(wl.pos, wl.mass, 295, targets=tg))


def test_knn_full_size_c2_sampled():
    # the 1,048,576-particle Plummer-cluster workload at the paper's K = 295, FP32 with the
    # radii estimated from the cell table (the bench launch configuration), checked on sampled
    # targets against the oracle's full sort
    wl = inputs.make("c2")
    g = gpu_knn(wl.pos, wl.mass, 295, 0.0, FP32)
    assert g["status"] == B.SPH_OK
    rng = np.random.default_rng(295)
    tg = np.sort(rng.choice(wl.n, size=96, replace=False))
    o = oracle.knn(wl.pos, wl.mass, 295, targets=tg, mode="brute")
    check_fp32(g, wl.pos, wl.mass, tg, 295, o)


def test_knn_after_batch_solve_needs_a_sort_and_graph_contexts_work():
    # kNN runs on the particles of sph_sort; a batched solve leaves groups, not one sorted set
    wl = inputs.make("c4", n_groups=8, nmax=256)
    s = B.Solver(wl.n, precision=FP32)
    s.batch_solve(T(wl.offsets, torch.int64), T(wl.pos), T(wl.mass), T(wl.h0), T(wl.nngb), T(wl.tol))
    h = torch.zeros(wl.n, dtype=torch.float64, device=DEV)
    rho = torch.empty_like(h)
    cnt = torch.empty(wl.n, dtype=torch.int32, device=DEV)
    assert B.sph_knn_solve(s.ctx, 16, h.data_ptr(), rho.data_ptr(), cnt.data_ptr()) == B.SPH_ERR_NOT_SORTED
    s.close()
    # a context whose density solves run as CUDA graphs: the kNN passes run from the host and
    # give the same answer
    u = inputs.make("c1", n=4096)
    ref = gpu_knn(u.pos, u.mass, 64, 0.0, FP64)
    s = B.Solver(u.n, precision=FP64, use_graph=True)
    s.sort(T(u.pos), T(u.mass))
    r = s.knn(64, torch.zeros(u.n, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    s.close()
    assert r["status"] == B.SPH_OK
    np.testing.assert_array_equal(r["h"].cpu().numpy(), ref["h"])
