"""O(N^2) brute-force neighbour sums in NumPy, used to pin the oracle's neighbour search.

For every target i and every particle j it forms the minimum-image separation (periodic)
or the plain separation, keeps the pairs with r < h_i (self included) and sums the M4
kernel.  It shares no code with the oracle or with the CUDA path.  The kernel shape is
written out again here, so this module pins the neighbour search, the periodic images and
the sums, not the kernel formula (the kernel is pinned by its own property tests).
"""
import math

import numpy as np


def _w(q):
    q = np.asarray(q, dtype=np.float64)
    inner = 1.0 - 6.0 * q * q + 6.0 * q * q * q
    a = 1.0 - q
    outer = 2.0 * a * a * a
    return np.where(q <= 0.5, inner, np.where(q < 1.0, outer, 0.0))


def _mqdw(q):
    q = np.asarray(q, dtype=np.float64)
    inner = 12.0 * q * q - 18.0 * q * q * q
    a = 1.0 - q
    outer = 6.0 * q * a * a
    return np.where(q <= 0.5, inner, np.where(q < 1.0, outer, 0.0))


def _w_c6(q):
    q = np.asarray(q, dtype=np.float64)
    a = np.clip(1.0 - q, 0.0, None)
    return a**8 * (1.0 + 8.0 * q + 25.0 * q * q + 32.0 * q**3)


def _mqdw_c6(q):
    q = np.asarray(q, dtype=np.float64)
    a = np.clip(1.0 - q, 0.0, None)
    return 22.0 * q * q * a**7 * (1.0 + 7.0 * q + 16.0 * q * q)


def evaluate(pos, mass, h, box=(1.0, 1.0, 1.0), periodic=True, targets=None, chunk=256, kernel="m4"):
    """rho, N_w, dN_w/dh, count for each target at its own h, by direct summation."""
    wf, dwf = (_w, _mqdw) if kernel == "m4" else (_w_c6, _mqdw_c6)
    sigma = 8.0 / math.pi if kernel == "m4" else 1365.0 / (64.0 * math.pi)
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    n = pos.shape[1]
    tg = np.arange(n) if targets is None else np.asarray(targets)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), tg.shape)
    box = np.asarray(box, dtype=np.float64)
    rho = np.empty(tg.shape[0])
    nw = np.empty(tg.shape[0])
    dnw = np.empty(tg.shape[0])
    count = np.empty(tg.shape[0], dtype=np.int64)
    for s in range(0, tg.shape[0], chunk):
        idx = tg[s:s + chunk]
        hh = h[s:s + chunk][:, None]
        d = pos[:, None, :] - pos[:, idx][:, :, None]  # (3, c, n): r_j - r_i
        if periodic:
            d = d - box[:, None, None] * np.round(d / box[:, None, None])
        r2 = (d * d).sum(axis=0)
        inside = r2 < hh * hh
        r = np.sqrt(r2)
        q = np.where(inside, r / hh, 1.0)
        w = np.where(inside, wf(q), 0.0)
        dw = np.where(inside, dwf(q), 0.0)
        hv = hh[:, 0]
        rho[s:s + chunk] = (w * mass[None, :]).sum(axis=1) * sigma / hv ** 3
        nw[s:s + chunk] = 4.0 * math.pi / 3.0 * sigma * w.sum(axis=1)
        dnw[s:s + chunk] = 4.0 * math.pi / 3.0 * sigma * dw.sum(axis=1) / hv
        count[s:s + chunk] = inside.sum(axis=1)
    return {"rho": rho, "nw": nw, "dnw": dnw, "count": count}


def neighbours(pos, h, targets, box=(1.0, 1.0, 1.0), periodic=True, band=0.0):
    """For each target i (at its own h_i), the particles j with r_ij < h_i (self included), and
    the particles with |r_ij - h_i| <= band * h_i with their FP64 distances r_ij (minimum image).

    Returns (inside, near): inside[k] is the sorted index array of target k's neighbours;
    near[k] is a dict {j: r_ij} of the pairs within the band around h."""
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    tg = np.asarray(targets)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), tg.shape)
    inside, near = [], []
    for k, i in enumerate(tg):
        d = pos - pos[:, i:i + 1]
        if periodic:
            d = d - box[:, None] * np.round(d / box[:, None])
        r2 = (d * d).sum(axis=0)
        hk = h[k]
        inside.append(np.flatnonzero(r2 < hk * hk))
        if band > 0.0:
            r = np.sqrt(r2)
            m = np.flatnonzero(np.abs(r - hk) <= band * hk)
            near.append({int(j): float(r[j]) for j in m})
        else:
            near.append({})
    return inside, near


def _mdw_over_q(q, kernel):
    """-w'(q)/q written from the shape polynomials (finite at q = 0)."""
    q = np.asarray(q, dtype=np.float64)
    if kernel == "m4":
        a = 1.0 - q
        outer = 6.0 * a * a / np.where(q > 0.0, q, 1.0)
        return np.where(q <= 0.5, 12.0 - 18.0 * q, np.where(q < 1.0, outer, 0.0))
    a = np.clip(1.0 - q, 0.0, None)
    return 22.0 * a**7 * (1.0 + 7.0 * q + 16.0 * q * q)


def interact(pos, mass, vel, h, box=(1.0, 1.0, 1.0), periodic=True, targets=None, kernel="m4", chunk=128):
    """Velocity mean, dispersion, divergence and curl over r < h_i by direct summation.

    Written in the shifted one-sweep form: with u_j = v_j - v_i, S0 = sum m W, S1 = sum m W u,
    S2 = sum m W |u|^2 give vmean = v_i + S1/S0 and sigma2 = S2/S0 - |S1/S0|^2; the kernel
    gradient is grad_i W = sigma g(q) (r_j - r_i) / h^5 with g = -w'(q)/q."""
    wf = _w if kernel == "m4" else _w_c6
    sigma = 8.0 / math.pi if kernel == "m4" else 1365.0 / (64.0 * math.pi)
    pos = np.asarray(pos, dtype=np.float64)
    vel = np.asarray(vel, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    n = pos.shape[1]
    tg = np.arange(n) if targets is None else np.asarray(targets)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), tg.shape)
    box = np.asarray(box, dtype=np.float64)
    T = tg.shape[0]
    out = {"rho": np.empty(T), "vmean": np.empty((3, T)), "sigma2": np.empty(T), "div": np.empty(T),
           "curl": np.empty((3, T)), "count": np.empty(T, dtype=np.int64)}
    for s in range(0, T, chunk):
        idx = tg[s:s + chunk]
        hh = h[s:s + chunk][:, None]
        d = pos[:, idx][:, :, None] - pos[:, None, :]  # (3, c, n): r_i - r_j
        if periodic:
            d = d - box[:, None, None] * np.round(d / box[:, None, None])
        r2 = (d * d).sum(axis=0)
        inside = r2 < hh * hh
        q = np.where(inside, np.sqrt(r2) / hh, 1.0)
        mW = np.where(inside, wf(q), 0.0) * mass[None, :] * sigma / hh ** 3
        mG = np.where(inside, _mdw_over_q(q, kernel), 0.0) * mass[None, :] * sigma / hh ** 5
        u = vel[:, None, :] - vel[:, idx][:, :, None]  # (3, c, n): v_j - v_i
        S0 = mW.sum(axis=1)
        S1 = (mW[None] * u).sum(axis=2)
        S2 = (mW * (u * u).sum(axis=0)).sum(axis=1)
        g = -mG[None] * d  # m_j grad_i W_ij, along r_j - r_i (W falls off with r)
        div = (u * g).sum(axis=0).sum(axis=1)
        cr = np.cross(-u, g, axis=0).sum(axis=2)  # (v_i - v_j) x m_j grad_i W_ij
        out["rho"][s:s + chunk] = S0
        mean_u = S1 / S0
        out["vmean"][:, s:s + chunk] = vel[:, idx] + mean_u
        out["sigma2"][s:s + chunk] = S2 / S0 - (mean_u * mean_u).sum(axis=0)
        out["div"][s:s + chunk] = div / S0
        out["curl"][:, s:s + chunk] = cr / S0
        out["count"][s:s + chunk] = inside.sum(axis=1)
    return out
