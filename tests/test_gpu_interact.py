"""The interaction pass (sph_interact) against the FP64 oracle: velocity mean, dispersion,
divergence and curl over each particle's neighbours at its h, the further pair computations
of the density loop (Listing 1).

Both sides get the same positions, masses, velocities and h (the GPU's converged h from a
density solve).  Tolerances follow from the arithmetic:
  - FP64 mode forms the neighbour test as the FP64 formulae do, so counts are exact; the sums
    differ from the oracle's only in rounding order and in the oracle taking the dispersion
    about the mean in a second sweep, so each output is held to ~1e-12 of its own scale:
    vscale2 = <|v_j - v_i|^2>_W for the dispersion, gabs = (1/rho) sum m |grad W| |v_j - v_i|
    for divergence and curl, |v| for the mean;
  - FP32 mode rounds velocities to FP32 (2^-24 of the largest component, vmax), offsets and
    pair terms to FP32 (compensated sums), and may decide pairs within 1e-6 h of the boundary
    either way (their kernel weight and gradient are below 1e-11 of a typical pair's).  So
    rho within 1e-5, the mean within 1e-5 sqrt(vscale2) + 1e-6 vmax, the dispersion within
    2e-5 vscale2 + 2e-6 vmax sqrt(vscale2), divergence and curl within 1e-5 gabs + 1e-6 vmax
    gnorm (gnorm = (1/rho) sum m |grad W|), counts within the pairs near the boundary.
"""
import numpy as np
import pytest

import oracle
from paper_1612_06090_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1612_06090_gb300 import binding as B  # noqa: E402

FP64, FP32 = B.SPH_PREC_FP64, B.SPH_PREC_FP32_KAHAN
DEV = torch.device("cuda:0")
KNAME = {B.SPH_KERNEL_M4: "m4", B.SPH_KERNEL_WENDLAND_C6: "wendland_c6"}


def T(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def gpu_interact(wl, vel, precision, kernel=B.SPH_KERNEL_M4, nngb=None, h=None):
    """Solve h on the GPU (unless given), then run the interaction pass at that h."""
    nngb = wl.nngb if nngb is None else nngb
    s = B.Solver(wl.n, precision=precision, box=wl.box, nngb=nngb, tol=wl.tol, kernel=kernel)
    s.sort(T(wl.pos), T(wl.mass))
    if h is None:
        r = s.solve(T(np.full(wl.n, inputs.mean_density_h(nngb, wl.n))))
        assert r["status"] == B.SPH_OK
        h = r["h"].cpu().numpy()
    out = s.interact(T(h), T(vel))
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    s.close()
    return h, g


def check(g, o, precision, near=None, tg=slice(None)):
    """GPU outputs g (rows tg) against oracle outputs o with the tolerances of the module doc."""
    vmax, vs2, gabs, gnorm = o["vmax"], o["vscale2"], o["gabs"], o["gnorm"]
    if precision == FP64:
        np.testing.assert_array_equal(g["count"][tg], o["count"])
        tr, tv, ts, td = 1e-12, 1e-12 * vmax, 1e-11 * vs2 + 1e-24 * vmax**2, 1e-11 * gabs
    else:
        dc = np.abs(g["count"][tg].astype(np.int64) - o["count"])
        assert np.all(dc <= near), int(np.max(dc - near))
        tr = 1e-5
        tv = 1e-5 * np.sqrt(vs2) + 1e-6 * vmax
        ts = 2e-5 * vs2 + 2e-6 * vmax * np.sqrt(vs2) + 1e-24 * vmax**2  # floor: a lone particle's
        # oracle dispersion is the rounding of its two-sweep mean, about 1e-33 v^2
        td = 1e-5 * gabs + 1e-6 * vmax * gnorm
    np.testing.assert_allclose(g["rho"][tg], o["rho"], rtol=tr)
    for name, tol in (("vmean", tv), ("curl", td)):
        err = np.abs(g[name][:, tg] - o[name])
        assert np.all(err <= tol), (name, float(np.max(err / tol)))
    for name, tol in (("sigma2", ts), ("div", td)):
        err = np.abs(g[name][tg] - o[name])
        assert np.all(err <= tol), (name, float(np.max(err / tol)))


@pytest.mark.parametrize("precision", [FP64, FP32])
@pytest.mark.parametrize("kernel,nngb", [(B.SPH_KERNEL_M4, 64.0), (B.SPH_KERNEL_WENDLAND_C6, 295.0)])
def test_uniform_box_against_oracle(precision, kernel, nngb):
    wl = inputs.make("c1")
    vel = inputs.velocities(wl.pos, 101)
    h, g = gpu_interact(wl, vel, precision, kernel, nngb)
    o = oracle.interact(wl.pos, wl.mass, vel, h, box=wl.box, kernel=KNAME[kernel])
    near = oracle.evaluate(wl.pos, wl.mass, h, box=wl.box, kernel=KNAME[kernel], near_rel=1e-6)["near"]
    check(g, o, precision, near)
    assert g["stats"]["pair_evals"] == int(g["count"].sum())
    assert g["stats"]["passes"] == 1


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_clustered_set_against_oracle(precision):
    # Plummer spheres + background: densities over orders of magnitude, items of every size
    wl = inputs.make("c2", n=1 << 17)
    vel = inputs.velocities(wl.pos, 102, bulk=2.0, sigma=0.1)
    h, g = gpu_interact(wl, vel, precision)
    o = oracle.interact(wl.pos, wl.mass, vel, h, box=wl.box)
    near = oracle.evaluate(wl.pos, wl.mass, h, box=wl.box, near_rel=1e-6)["near"]
    check(g, o, precision, near)


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_uniform_velocity_and_galilean_boost(precision):
    wl = inputs.make("c1", n=8192)
    c = np.array([2.5, -1.0, 0.75])
    h, g = gpu_interact(wl, np.repeat(c[:, None], wl.n, axis=1), precision)
    # every v_j - v_i is exactly zero: no divergence, curl or dispersion; the mean is v_i
    assert np.all(g["div"] == 0.0) and np.all(g["curl"] == 0.0) and np.all(g["sigma2"] == 0.0)
    np.testing.assert_array_equal(g["vmean"], np.repeat(c[:, None], wl.n, axis=1))
    vel = inputs.velocities(wl.pos, 103)
    _, a = gpu_interact(wl, vel, precision, h=h)
    _, b = gpu_interact(wl, vel + c[:, None], precision, h=h)
    o = oracle.interact(wl.pos, wl.mass, vel, h, box=wl.box)
    scale = 1e-12 if precision == FP64 else 1e-5
    np.testing.assert_array_equal(a["count"], b["count"])
    np.testing.assert_allclose(b["rho"], a["rho"], rtol=1e-15)
    vmax = np.abs(vel + c[:, None]).max()
    # FP32 rounds the boosted velocities anew: allow their rounding (2^-24 of the largest)
    extra = 0.0 if precision == FP64 else 4e-7 * vmax
    assert np.all(np.abs(b["vmean"] - c[:, None] - a["vmean"]) <= scale * np.sqrt(o["vscale2"]) + extra + 1e-13 * vmax)
    assert np.all(np.abs(b["sigma2"] - a["sigma2"]) <= 2 * scale * o["vscale2"] + 4 * extra * np.sqrt(o["vscale2"]))
    assert np.all(np.abs(b["div"] - a["div"]) <= 2 * scale * o["gabs"] + 2 * extra * o["gnorm"])


@pytest.mark.parametrize("n", [1, 2, 33, 257, 5003])
@pytest.mark.parametrize("precision", [FP64, FP32])
def test_ragged_sizes_and_anisotropic_box(n, precision):
    # fixed h (no solve): ragged particle counts, varied h, unequal masses, a non-cubic box
    rng = np.random.default_rng(500 + n)
    box = (1.0, 1.5, 0.75)
    pos = np.stack([rng.uniform(0, box[d], n) for d in range(3)])
    mass = rng.uniform(0.5, 2.0, n) / n
    vel = inputs.velocities(pos / np.array(box)[:, None], 106) + rng.normal(0.0, 0.1, (3, n))
    h = np.clip(inputs.mean_density_h(64.0, n / (box[0] * box[1] * box[2])) * rng.uniform(0.7, 1.3, n),
                1e-3, 0.37)
    s = B.Solver(n, precision=precision, box=box)
    s.sort(T(pos), T(mass))
    out = s.interact(T(h), T(vel))
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    s.close()
    o = oracle.interact(pos, mass, vel, h, box=box)
    near = oracle.evaluate(pos, mass, h, box=box, near_rel=1e-6)["near"]
    check(g, o, precision, near)


def test_errors_and_recovery():
    wl = inputs.make("c1")
    vel = inputs.velocities(wl.pos, 104)
    s = B.Solver(wl.n, precision=FP32, box=wl.box)
    h = T(wl.h0)
    # before any sort
    with pytest.raises(RuntimeError, match="NOT_SORTED|sort"):
        s.interact(h, T(vel))
    s.sort(T(wl.pos), T(wl.mass))
    L = B.lib()
    z = torch.zeros(3 * wl.n, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(wl.n, dtype=torch.int32, device=DEV)
    p = z.data_ptr()
    assert B.sph_interact(s.ctx, 0, p, p, p, p, p, p, cnt.data_ptr()) == B.SPH_ERR_INVALID_ARG
    assert B.sph_interact(s.ctx, h.data_ptr(), p, p, p, p, p, 0, cnt.data_ptr()) == B.SPH_ERR_INVALID_ARG
    assert L.sph_interact(None, None, None, None, None, None, None, None, None, None) == B.SPH_ERR_INVALID_ARG
    bad = vel.copy()
    bad[1, 17] = np.nan
    with pytest.raises(RuntimeError, match="velocity"):
        s.interact(h, T(bad))
    hb = wl.h0.copy()
    hb[5] = -1.0
    with pytest.raises(RuntimeError, match="DEVICE_STATUS|h not in"):
        s.interact(T(hb), T(vel))
    # the context still serves a valid call, equal to a fresh context's
    r = s.interact(h, T(vel))
    torch.cuda.synchronize()
    _, g = gpu_interact(wl, vel, FP32, h=wl.h0)
    np.testing.assert_array_equal(r["rho"].cpu().numpy(), g["rho"])
    np.testing.assert_array_equal(r["div"].cpu().numpy(), g["div"])
    s.close()


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_wendland_c6_clustered_against_oracle(precision):
    # the paper's kernel at 295 neighbours on Plummer spheres + background
    wl = inputs.make("c2", n=1 << 16, nngb=295.0, tol=5.0)
    vel = inputs.velocities(wl.pos, 107, bulk=1.5, sigma=0.2)
    h, g = gpu_interact(wl, vel, precision, B.SPH_KERNEL_WENDLAND_C6, 295.0)
    o = oracle.interact(wl.pos, wl.mass, vel, h, box=wl.box, kernel="wendland_c6")
    near = oracle.evaluate(wl.pos, wl.mass, h, box=wl.box, kernel="wendland_c6", near_rel=1e-6)["near"]
    check(g, o, precision, near)


def test_clumps_67M_sampled():
    # full size: snapshot 0 of the 67M-particle clump set at its FP32-converged h, sampled targets
    # against the oracle's brute force over every particle
    wl = inputs.make("c5")
    vel = inputs.velocities(wl.pos, 108)
    s = B.Solver(wl.n, precision=FP32, box=wl.box, nngb=wl.nngb, tol=wl.tol, use_graph=True)
    s.sort(T(wl.pos), T(wl.mass))
    r = s.solve(T(wl.h0))
    assert r["status"] == B.SPH_OK
    out = s.interact(r["h"], T(vel))
    torch.cuda.synchronize()
    g = {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in out.items()}
    h = r["h"].cpu().numpy()
    s.close()
    rng = np.random.default_rng(67)
    tg = np.sort(rng.choice(wl.n, size=32, replace=False))
    o = oracle.interact(wl.pos, wl.mass, vel, h[tg], box=wl.box, targets=tg, mode="brute")
    near = oracle.evaluate(wl.pos, wl.mass, h[tg], box=wl.box, targets=tg, mode="brute", near_rel=1e-6)["near"]
    check(g, o, FP32, near, tg)


def test_lognormal_16M_sampled():
    # full size: the 16.7M log-normal field (densities spanning orders of magnitude), FP32,
    # sampled targets against the oracle's brute force over every particle
    wl = inputs.make("c3")
    vel = inputs.velocities(wl.pos, 105)
    h, g = gpu_interact(wl, vel, FP32)
    rng = np.random.default_rng(33)
    tg = np.sort(rng.choice(wl.n, size=40, replace=False))
    o = oracle.interact(wl.pos, wl.mass, vel, h[tg], box=wl.box, targets=tg, mode="brute")
    near = oracle.evaluate(wl.pos, wl.mass, h[tg], box=wl.box, targets=tg, mode="brute", near_rel=1e-6)["near"]
    check(g, o, FP32, near, tg)
