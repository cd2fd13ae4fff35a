"""The seeded generators: deterministic, in range, with the structure each workload asks for."""
import hashlib

import numpy as np

from paper_1612_06090_gb300 import inputs


def _digest(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def test_uniform_is_deterministic_and_in_box():
    a = inputs.make("c1")
    b = inputs.make("c1")
    assert _digest(a.pos, a.mass, a.h0) == _digest(b.pos, b.mass, b.h0)
    assert a.pos.shape == (3, 4096) and a.pos.flags.c_contiguous
    assert np.all((a.pos >= 0) & (a.pos < 1))
    assert np.allclose(a.mass, 1 / 4096)
    assert np.allclose(a.h0, 0.15508762272485002, rtol=1e-15)


def test_plummer_clusters_small():
    wl = inputs.plummer_clusters(n=20000, seed=2)
    assert wl.pos.shape == (3, 20000)
    assert np.all((wl.pos >= 0) & (wl.pos < 1))
    assert wl.meta["n_clustered"] == 14000
    # clustered: the densest 1 % of a 32^3 grid holds far more than 1 % of the particles
    cells = np.floor(wl.pos * 32).astype(int)
    cid = cells[0] + 32 * (cells[1] + 32 * cells[2])
    counts = np.sort(np.bincount(cid, minlength=32**3))[::-1]
    assert counts[: 32**3 // 100].sum() > 0.3 * wl.n


def test_lognormal_small_has_voids():
    wl = inputs.lognormal_field(n=200000, seed=3, ng=32)
    assert np.all((wl.pos >= 0) & (wl.pos < 1))
    assert 0.02 < wl.meta["empty_cell_fraction"] < 0.6


def test_groups_offsets_and_sizes():
    wl = inputs.plummer_groups(n_groups=300, seed=4)
    sizes = np.diff(wl.offsets)
    assert wl.offsets[0] == 0 and wl.offsets[-1] == wl.n
    assert sizes.min() >= 32 and sizes.max() <= 200000
    assert np.all(wl.nngb == 32.0) and np.all(wl.tol == 1.0)
    # power law N^-2: the median size is about 2 * nmin
    assert 50 <= np.median(sizes) <= 90


def test_snapshots_share_particles_and_drift():
    s0 = inputs.clumpy_snapshots(n=40000, n_clumps=16, snapshot=0)
    s1 = inputs.clumpy_snapshots(n=40000, n_clumps=16, snapshot=1)
    d = s1.pos - s0.pos
    d -= np.round(d)
    assert 0.5e-4 < d.std() < 2e-4


def test_snapshot_series_matches_single_snapshots():
    from paper_1612_06090_gb300 import inputs as I

    series = list(I.clumpy_snapshot_series(3, n=20000, n_clumps=8))
    for s in range(3):
        one = I.clumpy_snapshots(n=20000, n_clumps=8, snapshot=s)
        np.testing.assert_array_equal(series[s].pos, one.pos)


def test_velocities_deterministic_periodic_and_scaled():
    import numpy as np

    rng = np.random.default_rng(3)
    pos = rng.uniform(0, 1, (3, 5000))
    a = inputs.velocities(pos, 11)
    b = inputs.velocities(pos, 11)
    np.testing.assert_array_equal(a, b)
    assert a.shape == (3, 5000) and np.all(np.isfinite(a))
    assert not np.array_equal(a, inputs.velocities(pos, 12))
    # the smooth part is continuous across the periodic faces: with the random part off, a shift
    # by one box length changes nothing (to rounding)
    s0 = inputs.velocities(pos, 11, sigma=0.0)
    s1 = inputs.velocities(pos + 1.0, 11, sigma=0.0)
    np.testing.assert_allclose(s0, s1, rtol=0, atol=1e-9)
    # rms of the smooth flow ~ bulk, of the random part ~ sigma
    assert 0.3 < np.sqrt(np.mean(s0**2) * 3) < 3.0
    r = inputs.velocities(pos, 11, bulk=0.0, sigma=0.3)
    assert abs(np.std(r) - 0.3) < 0.02
