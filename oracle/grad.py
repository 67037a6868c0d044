"""Plain FP64 CPU gradients of spectral functionals: the oracle of the
adjoint path.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the product never
imports it.

The paper's spectral projection (Sec. 2, Eq. XLXf) applied to f on a circle
with centre c and radius r, by the N-point trapezoid rule with the normalised
weights w_j = (z_j - c)/N, z_j = c + r e^{2πij/N}:

    x = P f ≈ Σ_j w_j x_j,   (A - z_j B) x_j = f,     Φ = ||x||².

Its derivative with respect to the entries of A and B follows from
dx_j = -(A - z_j B)^{-1} (dA - z_j dB) x_j:

    dΦ = -2 Re Σ_j μ_j^H (dA - z_j dB) x_j,   (A - z_j B)^H μ_j = conj(w_j) x,

so, for an entry (p, q) and the gradient convention g = ∂Φ/∂Re + i ∂Φ/∂Im,

    g_A[p,q] = -2 Σ_j μ_j[p] conj(x_j[q]),   g_B[p,q] = 2 Σ_j conj(z_j) μ_j[p] conj(x_j[q]).

For a simple eigenvalue λ with right and left eigenvectors x, y
(A x = λ B x, y^H A = λ y^H B) the derivative is dλ = y^H (dA - λ dB) x /
(y^H B x).  Both eigenvectors come from the same quadrature: x ∝ P v for a
random v, and y ∝ Σ_j conj(w_j) (A - z_j B)^{-H} B^H u for a random u (the
adjoint projector).  Every shifted system is solved by sparse LU.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def circle_nodes(c, r, N):
    """z_j = c + r e^{2πij/N} and the normalised trapezoid weights (z_j - c)/N."""
    ang = 2.0 * np.pi * np.arange(N) / N
    off = r * (np.cos(ang) + 1j * np.sin(ang))
    return c + off, off / N


def _B(A, B):
    n = A.shape[0]
    return sp.identity(n, dtype=np.complex128, format="csr") if B is None else sp.csr_matrix(B, dtype=np.complex128)


def projection_norm(A, B, f, c, r, N=16):
    """Φ = ||Σ_j w_j (A - z_j B)^{-1} f||² and the node solutions x_j."""
    A = sp.csr_matrix(A, dtype=np.complex128)
    Bm = _B(A, B)
    z, w = circle_nodes(c, r, N)
    X = np.array([spla.splu((A - zj * Bm).tocsc()).solve(np.asarray(f, dtype=np.complex128)) for zj in z])
    x = w @ X
    return float(np.vdot(x, x).real), x, X, z, w


def _entry_rows_cols(M):
    M = sp.csr_matrix(M)
    rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    return rows, M.indices


def projection_norm_grad(A, B, f, c, r, N=16):
    """Φ and its gradients on the stored entries of A (CSR order) and of B
    (None when B is the identity), convention ∂Φ/∂Re + i ∂Φ/∂Im."""
    A = sp.csr_matrix(A, dtype=np.complex128)
    Bm = _B(A, B)
    phi, x, X, z, w = projection_norm(A, B, f, c, r, N)
    Mu = np.array([spla.splu((A - zj * Bm).conj().T.tocsc()).solve(np.conj(wj) * x) for zj, wj in zip(z, w)])
    ra, ca = _entry_rows_cols(A)
    gA = -2.0 * np.einsum("je,je->e", Mu[:, ra], np.conj(X[:, ca]))
    gB = None
    if B is not None:
        rb, cb = _entry_rows_cols(Bm)
        gB = 2.0 * np.einsum("j,je,je->e", np.conj(z), Mu[:, rb], np.conj(X[:, cb]))
    return phi, gA, gB


def eigenvalue_grad(A, B, c, r, N=16, seed=0):
    """A simple eigenvalue λ inside the circle (c, r) — the Rayleigh quotient
    y^H A x / y^H B x of the quadrature eigenvectors — and dλ/dA, dλ/dB on
    the stored entries (CSR order; dλ/dB None when B is the identity)."""
    A = sp.csr_matrix(A, dtype=np.complex128)
    Bm = _B(A, B)
    n = A.shape[0]
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    z, w = circle_nodes(c, r, N)
    x = np.zeros(n, dtype=np.complex128)
    y = np.zeros(n, dtype=np.complex128)
    for zj, wj in zip(z, w):
        K = (A - zj * Bm).tocsc()
        x += wj * spla.splu(K).solve(v)
        y += np.conj(wj) * spla.splu(K.conj().T.tocsc()).solve(Bm.conj().T @ u)
    yBx = np.vdot(y, Bm @ x)
    lam = np.vdot(y, A @ x) / yBx
    ra, ca = _entry_rows_cols(A)
    dA = np.conj(y[ra]) * x[ca] / yBx
    dB = None
    if B is not None:
        rb, cb = _entry_rows_cols(Bm)
        dB = -lam * np.conj(y[rb]) * x[cb] / yBx
    return complex(lam), dA, dB
