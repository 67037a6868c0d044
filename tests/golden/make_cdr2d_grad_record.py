"""Writes cdr2d500_grad_record.json: oracle gradients (oracle/grad.py, sparse
LU at every node) on the n = 250,000 convection–diffusion–reaction workload:
Φ = ||P f||² on a circle around the lowest eigenvalue and its gradient, the
eigenvalue and dλ/dA, each on 32 sampled diagonal entries (the reaction
coefficients).  Calls only the oracle and the seeded workload generators.

    python tests/golden/make_cdr2d_grad_record.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import grad as G  # noqa: E402
from workloads import cdr_separable_eigenvalues  # noqa: E402
from workloads.configs import config_cdr2d  # noqa: E402

N_GRID = 500
SAMPLE_SEED = 7


def circle():
    """Centre 0.5 right of the smallest separable eigenvalue (the reaction
    0 <= c <= 1 moves each eigenvalue right by at most 1), radius 3: the
    next eigenvalue lies about 30 further right."""
    lam0 = float(np.min(cdr_separable_eigenvalues((N_GRID, N_GRID), (1.0, 0.5)).real))
    return complex(lam0 + 0.5, 0.0), 3.0


def sample_entries(A):
    """32 diagonal entries (row, position in A's CSR arrays)."""
    M = A.to_scipy()
    rows = np.sort(np.random.default_rng(SAMPLE_SEED).choice(M.shape[0], 32, replace=False))
    pos = np.array([M.indptr[r] + int(np.nonzero(M.indices[M.indptr[r]:M.indptr[r + 1]] == r)[0][0]) for r in rows])
    return rows, pos


def main():
    w = config_cdr2d(N_GRID)
    c, r = circle()
    rows, pos = sample_entries(w.A)
    t0 = time.time()
    phi, gA, _ = G.projection_norm_grad(w.A.to_scipy(), None, w.f, c, r, 16)
    lam, dA, _ = G.eigenvalue_grad(w.A.to_scipy(), None, c, r, 16)
    out = dict(
        workload=w.name, center=[c.real, c.imag], radius=r, nodes=16,
        phi=phi, lam=[lam.real, lam.imag],
        rows=[int(x) for x in rows], positions=[int(x) for x in pos],
        grad_phi_re=[float(x) for x in gA[pos].real], grad_phi_im=[float(x) for x in gA[pos].imag],
        dlam_re=[float(x) for x in dA[pos].real], dlam_im=[float(x) for x in dA[pos].imag],
        oracle_seconds=round(time.time() - t0, 1),
    )
    with open(os.path.join(HERE, "cdr2d500_grad_record.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("phi", phi, "lam", lam, "%.1fs" % out["oracle_seconds"])


if __name__ == "__main__":
    main()
