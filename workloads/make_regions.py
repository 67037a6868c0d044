"""Writes ``regions.json``: search regions for pencils without a closed-form
spectrum, placed by exact inertia counts (the oracle's Sylvester-inertia
counter).  Run from the repository root:  python -m workloads.make_regions

pencil200: the 200×200 convection–diffusion operator with B = diag(U[1,2])
(seed 1).  The region's real edges are the midpoints of the gaps below
λ_k0 and above λ_{k0+499}, k0 = 19750 (mid-spectrum, 500 eigenvalues);
Im range [-0.3, 0.7].
"""
from __future__ import annotations

import json
import os

from oracle.inertia import count_below, kth_eigenvalue_bracket
from workloads.configs import pencil_parts


def edge_between(N, beta, bd, k, lo, hi):
    """Midpoint between λ_{k-1} and λ_k (0-based ascending)."""
    a = kth_eigenvalue_bracket(N, beta, bd, k - 1, lo, hi, 1e-4)
    b = kth_eigenvalue_bracket(N, beta, bd, k, a[0], hi, 1e-4)
    return 0.5 * (a[1] + b[0]), b[0] - a[1]


def main():
    N, beta = 200, (1.0, 0.5)
    _, bd = pencil_parts(N, 1)
    k0, cnt = 19750, 500
    lo_all, hi_all = 0.0, 8.0 * (N + 1) ** 2 + 10.0
    re_lo, gap_lo = edge_between(N, beta, bd, k0, lo_all, hi_all)
    re_hi, gap_hi = edge_between(N, beta, bd, k0 + cnt, re_lo, hi_all)
    got = count_below(N, beta, bd, re_hi) - count_below(N, beta, bd, re_lo)
    assert got == cnt, got
    out = {"pencil200": {"region": [re_lo, re_hi, -0.3, 0.7], "count": cnt,
                          "k0": k0, "edge_gaps": [gap_lo, gap_hi]}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "regions.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    main()
