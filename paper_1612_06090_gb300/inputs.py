"""Seeded synthetic particle sets for the SPH density / smoothing-length solve.

This module only draws positions, masses, starting smoothing lengths and (for the
interaction pass) velocities.  It holds
none of the method's arithmetic (no kernel, no neighbour search, no h update), so both
the CUDA path and the FP64 oracle may take their inputs from it.

The paper's own workload is a serialised P-Gadget3 snapshot of 81^3 dark-matter and
81^3 gas particles (Sec. II-C); it is not available, so these generators stand in for it
with the shapes and density contrasts of the five benchmark configurations:

  c1  4,096 uniform particles in the periodic unit box, Nngb = 64 +- 2.
  c2  1,048,576 particles: 70 % in 64 Plummer spheres (a = 0.01) + 30 % uniform.
  c3  16,777,216 particles drawn from a log-normal density field (64^3 grid,
      P(k) ~ k^-2, sigma_ln = 2), jittered within grid cells.
  c4  20,000 independent non-periodic Plummer groups (a = 1), sizes from
      dN/dN ~ N^-2 on [32, 200000], Nngb = 32 +- 1 per group.
  c5  67,108,864 particles: 4,096 Plummer clumps (70 %, a log-uniform in
      [1e-3, 1e-2]) + uniform background; snapshots drift by N(0, 1e-4^2).

Every array is float64.  Positions come as a (3, N) array (x, y, z planes), which is
the layout the C ABI takes.  Equal masses 1/N.  The starting smoothing length is the
one that encloses Nngb neighbours at the mean density, h0 = (3 Nngb / (4 pi n))^(1/3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "BatchWorkload",
    "uniform_box",
    "plummer_clusters",
    "lognormal_field",
    "plummer_groups",
    "clumpy_snapshots",
    "clumpy_snapshot_series",
    "make",
    "velocities",
    "mean_density_h",
    "CONFIG_SEEDS",
]

# Seeds are the configuration number, so every run draws the same particles.
CONFIG_SEEDS = {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5}


@dataclass
class Workload:
    """One periodic particle set."""

    name: str
    pos: np.ndarray  # (3, N) float64, each coordinate in [0, box[d])
    mass: np.ndarray  # (N,) float64
    h0: np.ndarray  # (N,) float64 starting smoothing lengths
    box: tuple = (1.0, 1.0, 1.0)
    periodic: bool = True
    nngb: float = 64.0
    tol: float = 2.0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])


@dataclass
class BatchWorkload:
    """Many independent non-periodic groups, flattened group after group."""

    name: str
    offsets: np.ndarray  # (G+1,) int64, group g is [offsets[g], offsets[g+1])
    pos: np.ndarray  # (3, N) float64
    mass: np.ndarray  # (N,) float64
    h0: np.ndarray  # (N,) float64
    nngb: np.ndarray  # (G,) float64
    tol: np.ndarray  # (G,) float64
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.mass.shape[0])

    @property
    def n_groups(self) -> int:
        return int(self.offsets.shape[0] - 1)


def mean_density_h(nngb: float, number_density: float) -> float:
    """Radius of the sphere that holds nngb particles at the given number density."""
    return (3.0 * nngb / (4.0 * math.pi * number_density)) ** (1.0 / 3.0)


def _wrap(pos: np.ndarray, box) -> np.ndarray:
    """Wrap each coordinate plane into [0, box[d])."""
    out = np.empty_like(pos)
    for d in range(3):
        L = float(box[d])
        v = np.mod(pos[d], L)
        # np.mod can return L itself for tiny negative inputs; fold that back to 0.
        v[v >= L] = 0.0
        out[d] = v
    return out


def _plummer_offsets(rng: np.random.Generator, n: int, a: float, rmax_over_a: float) -> np.ndarray:
    """Offsets (3, n) of Plummer-sphere particles with scale radius a, truncated at rmax.

    The enclosed mass fraction of a Plummer sphere is X = r^3 / (r^2 + a^2)^(3/2), so
    r = a / sqrt(X^(-2/3) - 1).  Truncation draws X uniformly below X(rmax).
    """
    xmax = rmax_over_a**3 / (rmax_over_a**2 + 1.0) ** 1.5
    X = rng.uniform(0.0, xmax, size=n)
    X = np.maximum(X, 1e-300)
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    # isotropic directions
    cos_t = rng.uniform(-1.0, 1.0, size=n)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    return np.stack([r * sin_t * np.cos(phi), r * sin_t * np.sin(phi), r * cos_t])


def _split_counts(total: int, parts: int) -> np.ndarray:
    """Split total into `parts` counts that differ by at most one."""
    base = total // parts
    counts = np.full(parts, base, dtype=np.int64)
    counts[: total - base * parts] += 1
    return counts


def uniform_box(n: int = 4096, seed: int = 1, nngb: float = 64.0, tol: float = 2.0,
                box=(1.0, 1.0, 1.0)) -> Workload:
    """Config c1: n uniform particles in a periodic box, equal masses 1/n."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    pos = np.stack([rng.uniform(0.0, box[d], size=n) for d in range(3)])
    pos = _wrap(pos, box)
    vol = float(box[0]) * float(box[1]) * float(box[2])
    h0 = np.full(n, mean_density_h(nngb, n / vol))
    return Workload("uniform", np.ascontiguousarray(pos), np.full(n, 1.0 / n), h0,
                    tuple(float(b) for b in box), True, nngb, tol,
                    {"seed": seed, "recipe": "uniform random in the periodic box"})


def plummer_clusters(n: int = 1 << 20, seed: int = 2, n_spheres: int = 64, a: float = 0.01,
                     frac: float = 0.7, trunc: float = 50.0, nngb: float = 64.0,
                     tol: float = 2.0) -> Workload:
    """Config c2: n_spheres Plummer spheres (70 % of the particles) + uniform background.

    Sphere centres are uniform random; each sphere holds an equal share (counts differ by
    at most one); radii are truncated at `trunc` * a and positions wrap periodically.
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    n_cl = int(round(frac * n))
    counts = _split_counts(n_cl, n_spheres)
    centres = rng.uniform(0.0, 1.0, size=(n_spheres, 3))
    parts = []
    for s in range(n_spheres):
        off = _plummer_offsets(rng, int(counts[s]), a, trunc)
        parts.append(off + centres[s][:, None])
    bg = rng.uniform(0.0, 1.0, size=(3, n - n_cl))
    pos = _wrap(np.concatenate(parts + [bg], axis=1), (1.0, 1.0, 1.0))
    # shuffle so that caller order carries no spatial structure
    perm = rng.permutation(n)
    pos = np.ascontiguousarray(pos[:, perm])
    h0 = np.full(n, mean_density_h(nngb, float(n)))
    return Workload("plummer64", pos, np.full(n, 1.0 / n), h0, (1.0, 1.0, 1.0), True, nngb, tol,
                    {"seed": seed, "n_spheres": n_spheres, "a": a, "frac": frac,
                     "truncation_radius_over_a": trunc, "n_clustered": n_cl})


def _gaussian_field(rng: np.random.Generator, ng: int, slope: float) -> np.ndarray:
    """Real Gaussian random field on an ng^3 grid with power spectrum P(k) ~ k^slope.

    White noise is filtered in Fourier space by sqrt(P(k)); the k = 0 mode is zeroed and
    the result is normalised to zero mean and unit standard deviation.
    """
    white = rng.standard_normal((ng, ng, ng))
    wk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(ng) * ng
    kz = np.fft.rfftfreq(ng) * ng
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # sqrt(P) with P ~ k^slope = (k^2)^(slope/2)
    g = np.fft.irfftn(wk * amp, s=(ng, ng, ng), axes=(0, 1, 2))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_field(n: int = 1 << 24, seed: int = 3, ng: int = 64, slope: float = -2.0,
                    sigma_ln: float = 2.0, nngb: float = 64.0, tol: float = 2.0) -> Workload:
    """Config c3: particles sampled from a log-normal density field.

    ln rho = sigma_ln * g - sigma_ln^2 / 2 (mean one) on an ng^3 grid; cell counts are
    multinomial(n, rho / sum rho) and each particle is placed uniformly inside its cell.
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    g = _gaussian_field(rng, ng, slope)
    rho = np.exp(sigma_ln * g - 0.5 * sigma_ln * sigma_ln)
    p = (rho / rho.sum()).ravel()
    counts = rng.multinomial(n, p)
    cell = np.repeat(np.arange(ng**3, dtype=np.int64), counts)
    ix = cell // (ng * ng)
    iy = (cell // ng) % ng
    iz = cell % ng
    c = 1.0 / ng
    pos = np.stack([(ix + rng.uniform(0.0, 1.0, n)) * c,
                    (iy + rng.uniform(0.0, 1.0, n)) * c,
                    (iz + rng.uniform(0.0, 1.0, n)) * c])
    pos = _wrap(pos, (1.0, 1.0, 1.0))
    perm = rng.permutation(n)
    pos = np.ascontiguousarray(pos[:, perm])
    h0 = np.full(n, mean_density_h(nngb, float(n)))
    return Workload("lognormal", pos, np.full(n, 1.0 / n), h0, (1.0, 1.0, 1.0), True, nngb, tol,
                    {"seed": seed, "grid": ng, "slope": slope, "sigma_ln": sigma_ln,
                     "empty_cell_fraction": float(np.mean(counts == 0))})


def _powerlaw_sizes(rng: np.random.Generator, n_groups: int, nmin: int, nmax: int,
                    alpha: float) -> np.ndarray:
    """Group sizes with dN/dN ~ N^-alpha on [nmin, nmax] by inverse CDF, rounded."""
    u = rng.uniform(0.0, 1.0, size=n_groups)
    if abs(alpha - 1.0) < 1e-12:
        s = nmin * (nmax / nmin) ** u
    else:
        e = 1.0 - alpha
        s = (nmin**e + u * (nmax**e - nmin**e)) ** (1.0 / e)
    return np.clip(np.rint(s).astype(np.int64), nmin, nmax)


def plummer_groups(n_groups: int = 20000, seed: int = 4, nmin: int = 32, nmax: int = 200000,
                   alpha: float = 2.0, a: float = 1.0, trunc: float = 20.0, nngb: float = 32.0,
                   tol: float = 1.0) -> BatchWorkload:
    """Config c4: independent non-periodic Plummer groups of power-law sizes.

    The starting h of a group is the Nngb-sphere radius at the group's mean number density
    inside its half-mass radius (of the truncated sphere).
    """
    rng = np.random.default_rng(np.random.PCG64(seed))
    sizes = _powerlaw_sizes(rng, n_groups, nmin, nmax, alpha)
    offsets = np.zeros(n_groups + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    n = int(offsets[-1])
    pos = np.empty((3, n))
    h0 = np.empty(n)
    mass = np.empty(n)
    xmax = trunc**3 / (trunc**2 + 1.0) ** 1.5
    xhalf = 0.5 * xmax
    r_half = a / math.sqrt(xhalf ** (-2.0 / 3.0) - 1.0)
    for g in range(n_groups):
        s, e = int(offsets[g]), int(offsets[g + 1])
        k = e - s
        pos[:, s:e] = _plummer_offsets(rng, k, a, trunc)
        dens = 0.5 * k / (4.0 / 3.0 * math.pi * r_half**3)
        h0[s:e] = mean_density_h(nngb, dens)
        mass[s:e] = 1.0 / k
    return BatchWorkload("plummer_groups", offsets, np.ascontiguousarray(pos), mass, h0,
                         np.full(n_groups, float(nngb)), np.full(n_groups, float(tol)),
                         {"seed": seed, "alpha": alpha, "nmin": nmin, "nmax": nmax,
                          "a": a, "truncation_radius_over_a": trunc, "total": n})


def _parallel(fn, items):
    """Run fn over items on a thread pool (NumPy's generators and ufuncs release the GIL)."""
    import concurrent.futures
    import os

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        list(ex.map(fn, items))


_CHUNK = 1 << 22


def _wrap_unit_inplace(pos: np.ndarray) -> None:
    """Wrap every coordinate of a (3, n) array into [0, 1) in place (chunked, threaded).

    x - floor(x) equals np.mod(x, 1.0) for the |x| < 2 that occur here; a tiny negative x
    can round up to 1.0, which folds back to 0 as in _wrap."""
    flat = pos.reshape(-1)

    def one(k):
        v = flat[k:k + _CHUNK]
        v -= np.floor(v)
        v[v >= 1.0] = 0.0

    _parallel(one, range(0, flat.size, _CHUNK))


def _add_drift_inplace(pos: np.ndarray, seed: int, step: int, drift: float) -> None:
    """Add drift step `step` (>= 1): N(0, drift^2) per coordinate, drawn in chunks of 2^22
    values from independent PCG64 streams seeded by (seed, step, chunk)."""
    flat = pos.reshape(-1)

    def one(k):
        g = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 17, step, k // _CHUNK])))
        v = flat[k:k + _CHUNK]
        d = g.standard_normal(size=v.shape[0])
        d *= drift
        v += d

    _parallel(one, range(0, flat.size, _CHUNK))


def _clumpy_base(n, seed, n_clumps, a_range, frac, trunc):
    """Unwrapped snapshot-0 positions of config c5 (a fresh (3, n) array)."""
    rng = np.random.default_rng(np.random.PCG64(seed))
    n_cl = int(round(frac * n))
    counts = _split_counts(n_cl, n_clumps)
    centres = rng.uniform(0.0, 1.0, size=(n_clumps, 3))
    radii = np.exp(rng.uniform(math.log(a_range[0]), math.log(a_range[1]), size=n_clumps))
    pos = np.empty((3, n))
    o = 0
    for c in range(n_clumps):
        k = int(counts[c])
        pos[:, o:o + k] = _plummer_offsets(rng, k, float(radii[c]), trunc) + centres[c][:, None]
        o += k
    pos[:, n_cl:] = rng.uniform(0.0, 1.0, size=(3, n - n_cl))
    perm = rng.permutation(n)
    out = np.empty_like(pos)

    def gather(d):
        np.take(pos[d], perm, out=out[d])

    _parallel(gather, range(3))
    return out


def clumpy_snapshot_series(n_snapshots: int = 8, n: int = 1 << 26, seed: int = 5, n_clumps: int = 4096,
                           a_range=(1e-3, 1e-2), frac: float = 0.7, trunc: float = 50.0,
                           drift: float = 1e-4, nngb: float = 64.0, tol: float = 2.0, first: int = 0):
    """Yield snapshots first .. n_snapshots-1 of config c5 one after another.

    Config c5: Plummer clumps (70 % of the particles, log-uniform scale radii, truncated at
    `trunc` scale radii) + a uniform background in the periodic unit box.  Snapshot s adds s
    independent N(0, drift^2) steps per coordinate to snapshot 0 and wraps; snapshots share
    the same particle identities, so an h solved on snapshot s-1 is a warm start for
    snapshot s.  Each yielded Workload owns its position array.
    """
    base = _clumpy_base(n, seed, n_clumps, a_range, frac, trunc)
    mass = np.full(n, 1.0 / n)
    h0 = np.full(n, mean_density_h(nngb, float(n)))
    meta = {"seed": seed, "n_clumps": n_clumps, "a_range": list(a_range), "drift": drift,
            "n_snapshots": n_snapshots}
    for s in range(n_snapshots):
        if s > 0:
            _add_drift_inplace(base, seed, s, drift)
        if s < first:
            continue
        pos = base.copy()
        _wrap_unit_inplace(pos)
        yield Workload("clumps4096", pos, mass, h0, (1.0, 1.0, 1.0), True, nngb, tol, {**meta, "snapshot": s})


def clumpy_snapshots(snapshot: int = 0, **kw) -> Workload:
    """Config c5, snapshot `snapshot` alone (the same particles as clumpy_snapshot_series)."""
    kw.setdefault("n_snapshots", max(8, snapshot + 1))
    n_snap = kw.pop("n_snapshots")
    for wl in clumpy_snapshot_series(n_snapshots=n_snap, first=snapshot, **kw):
        wl.meta["n_snapshots"] = n_snap
        return wl
    raise ValueError(f"snapshot {snapshot} outside the series")


def velocities(pos: np.ndarray, seed: int, bulk: float = 1.0, sigma: float = 0.3, n_modes: int = 6,
               kmax: int = 3) -> np.ndarray:
    """Seeded synthetic velocities for the interaction pass, (3, N) float64.

    A smooth periodic flow, sum of n_modes Fourier modes a_m sin(2 pi k_m . x + phi_m) with
    integer wave vectors |k_m,d| <= kmax (continuous across the periodic faces of the unit
    box) and amplitudes N(0, bulk^2 / n_modes) per component, plus independent N(0, sigma^2)
    per component and particle (the local dispersion).  The stream of draws depends on seed
    only.
    """
    rng = np.random.default_rng(np.random.PCG64([seed, 23]))
    k = rng.integers(-kmax, kmax + 1, size=(n_modes, 3)).astype(np.float64)
    k[np.all(k == 0, axis=1), 0] = 1.0
    amp = rng.normal(0.0, bulk / math.sqrt(n_modes), size=(n_modes, 3))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=(n_modes, 3))
    n = pos.shape[1]
    vel = np.empty((3, n))

    def one(c0):
        c1 = min(n, c0 + _CHUNK)
        x = pos[:, c0:c1]
        g = np.random.default_rng(np.random.PCG64([seed, 29, c0 // _CHUNK]))
        out = g.normal(0.0, sigma, size=(3, c1 - c0))
        for m in range(n_modes):
            arg = 2.0 * math.pi * (k[m] @ x)
            for d in range(3):
                out[d] += amp[m, d] * np.sin(arg + phase[m, d])
        vel[:, c0:c1] = out

    _parallel(one, range(0, n, _CHUNK))
    return vel


def make(config: str, **kw):
    """Build a named configuration (c1..c5) with optional overrides (e.g. n=...)."""
    config = config.lower()
    if config == "c1":
        return uniform_box(**{"seed": CONFIG_SEEDS["c1"], **kw})
    if config == "c2":
        return plummer_clusters(**{"seed": CONFIG_SEEDS["c2"], **kw})
    if config == "c3":
        return lognormal_field(**{"seed": CONFIG_SEEDS["c3"], **kw})
    if config == "c4":
        return plummer_groups(**{"seed": CONFIG_SEEDS["c4"], **kw})
    if config == "c5":
        return clumpy_snapshots(**{"seed": CONFIG_SEEDS["c5"], **kw})
    raise ValueError(f"unknown configuration {config!r}")
