"""Exact eigenvalue counts for the convection–diffusion pencils by Sylvester's
law of inertia.

TEST INFRASTRUCTURE ONLY (part of the oracle; independent of SIM-M).

The 5-point operator A = T_x ⊗ I + I ⊗ T_y with tridiagonal Toeplitz factors
T = tridiag(b, a, c), bc > 0, is similar to the symmetric S = D^{-1} A D with
the diagonal D = D_y ⊗ D_x, (D_x)_ii = (b/c)^{i/2}.  A diagonal B commutes with
D, so the pencil (A, B) is similar to the symmetric-definite (S, B) and all its
eigenvalues are real.  The number below x equals the number of negative
eigenvalues of S - xB, which block LDL^T (Schur complements D_k of the block
tridiagonal S - xB) gives as Σ_k #neg(D_k) (Haynsworth inertia additivity).
"""
from __future__ import annotations

import numpy as np


def _sym_factor(N, b):
    h = 1.0 / (N + 1)
    prod = (1.0 / h**2 + b / (2 * h)) * (1.0 / h**2 - b / (2 * h))
    return 2.0 / h**2, -np.sqrt(prod)


def count_below(N: int, beta, bdiag, x: float) -> int:
    """#{λ < x} for the pencil (cd2d(N, beta), diag(bdiag)), bdiag > 0."""
    ax, ox = _sym_factor(N, float(beta[0]))
    ay, oy = _sym_factor(N, float(beta[1]))
    bdiag = np.asarray(bdiag, dtype=np.float64).reshape(N, N)  # [iy, ix]
    Sx = np.diag(np.full(N, ax + ay)) + np.diag(np.full(N - 1, ox), 1) + np.diag(np.full(N - 1, ox), -1)
    neg = 0
    Dinv = None
    for k in range(N):
        Dk = Sx - x * np.diag(bdiag[k])
        if Dinv is not None:
            Dk = Dk - (oy * oy) * Dinv
        Dk = 0.5 * (Dk + Dk.T)
        w = np.linalg.eigvalsh(Dk)
        neg += int(np.sum(w < 0))
        Dinv = np.linalg.inv(Dk)
    return neg


def kth_eigenvalue_bracket(N, beta, bdiag, k, lo, hi, tol):
    """Bisection for λ_k (0-based, ascending): returns (a, b) with
    count_below(a) <= k < count_below(b) and b - a <= tol."""
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if count_below(N, beta, bdiag, mid) <= k:
            lo = mid
        else:
            hi = mid
    return lo, hi
