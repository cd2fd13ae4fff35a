"""Write lattice16.json: the density of a simple cubic lattice by lattice-vector enumeration.

A 16^3 simple cubic lattice of spacing s = 1/16 fills the periodic unit box with masses
1/4096.  Every particle sees the same neighbourhood, so its density is a lattice sum
over integer vectors v = (i, j, k) with |v| s < h:
    rho = m * 8 / (pi h^3) * sum_v w(|v| s / h),   N_w = (32/3) sum_v w(|v| s / h),
    n   = #{v : |v| s < h}.
This script enumerates the vectors directly (no grid, no periodic images: h < 1/2) and
takes w from the oracle, whose shape is pinned by its own property tests.  The root of
N_w(h) = 64 is found by bisection on the lattice sum.  Only oracle/ is called.

Run from the repository root:  python tests/golden/make_lattice_golden.py
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

S = 1.0 / 16.0
M = 1.0 / 4096.0
H0 = (3.0 * 64.0 / (4.0 * math.pi * 4096.0)) ** (1.0 / 3.0)


def lattice_sums(h):
    kmax = int(math.ceil(h / S)) + 1
    sw = 0.0
    n = 0
    # sum the smallest terms first: group vectors by |v|^2
    shells = {}
    for i in range(-kmax, kmax + 1):
        for j in range(-kmax, kmax + 1):
            for k in range(-kmax, kmax + 1):
                r2 = (i * i + j * j + k * k)
                if r2 * S * S < h * h:
                    shells[r2] = shells.get(r2, 0) + 1
    for r2 in sorted(shells, reverse=True):
        q = math.sqrt(r2) * S / h
        sw += shells[r2] * oracle.w(q)
        n += shells[r2]
    return M * 8.0 / (math.pi * h ** 3) * sw, 32.0 / 3.0 * sw, n


def main():
    rho, nw, n = lattice_sums(H0)
    lo, hi = H0, H0 * 1.01
    assert lattice_sums(lo)[1] < 64.0 < lattice_sums(hi)[1]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if lattice_sums(mid)[1] < 64.0:
            lo = mid
        else:
            hi = mid
    out = {
        "what": "16^3 simple cubic lattice, periodic unit box, m = 1/4096, M4 kernel",
        "how": "direct enumeration of lattice vectors (tests/golden/make_lattice_golden.py)",
        "h0": H0,
        "rho_at_h0": rho,
        "nw_at_h0": nw,
        "count_at_h0": n,
        "root_nw_64": 0.5 * (lo + hi),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice16.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
