"""Pins for the oracle gradients (oracle/grad.py): closed forms for a
diagonal matrix, central finite differences, and the invariances of a simple
eigenvalue (shift, homogeneity, joint scaling of A and B)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import grad as G
from workloads import cdr_csr, complex_gaussian, diag_csr


def _perturb(M, e, delta):
    M = sp.csr_matrix(M, dtype=np.complex128, copy=True)
    M.data[e] += delta
    return M


def _small_pencil(seed=0, general_B=False):
    """A non-normal 2-D convection–diffusion–reaction pencil (n = 42) with a
    diagonal or a general (tridiagonal, diagonally dominant) B."""
    rng = np.random.default_rng(seed)
    A = cdr_csr((7, 6), (3.0, -2.0), rng.uniform(0, 1, 42) + 0.3j * rng.uniform(-1, 1, 42)).to_scipy()
    if general_B:
        B = sp.diags([0.1 * rng.standard_normal(41), 1.5 + rng.uniform(0, 0.5, 42), 0.1 * rng.standard_normal(41)],
                     [-1, 0, 1], format="csr", dtype=np.complex128)
    else:
        B = sp.diags(rng.uniform(1, 2, 42), format="csr", dtype=np.complex128)
    return A, B


def test_projection_norm_closed_form_diagonal():
    lam = np.array([1.0 + 0.2j, 1.3 - 0.1j, 0.7 + 0.5j, 4.0 + 4.0j, -2.0 + 0.0j])
    f = complex_gaussian(lam.size, 3)
    c, r, N = 1.0 + 0.1j, 0.6, 16
    phi, gA, _ = G.projection_norm_grad(diag_csr(lam).to_scipy(), None, f, c, r, N)
    u = (lam - c) / r
    g = 1 - u**N
    # trapezoid identity: Σ_j w_j/(λ - z_j) = -1/(1 - u^N)
    assert abs(phi - np.sum(np.abs(f) ** 2 / np.abs(g) ** 2)) <= 1e-12 * phi
    # Wirtinger: 2 ∂Φ/∂conj(λ_k) = 2|f_k|² N g conj(u^{N-1}) / (r |g|^4)
    want = 2 * np.abs(f) ** 2 * N * g * np.conj(u ** (N - 1)) / (r * np.abs(g) ** 4)
    assert np.max(np.abs(gA - want)) <= 1e-10 * np.max(np.abs(want))


@pytest.mark.parametrize("general_B", [False, True])
def test_projection_norm_grad_central_differences(general_B):
    A, B = _small_pencil(1, general_B)
    f = complex_gaussian(A.shape[0], 4)
    c, r = 40.0 + 0.2j, 25.0
    phi, gA, gB = G.projection_norm_grad(A, B, f, c, r)
    rng = np.random.default_rng(2)
    h = 1e-6
    for M, grad, which in ((A, gA, "A"), (B, gB, "B")):
        for e in rng.choice(M.nnz, 6, replace=False):
            for part in (1.0, 1j):
                Ap, Bp = (_perturb(A, e, h * part), B) if which == "A" else (A, _perturb(B, e, h * part))
                Am, Bm = (_perturb(A, e, -h * part), B) if which == "A" else (A, _perturb(B, e, -h * part))
                fd = (G.projection_norm(Ap, Bp, f, c, r)[0] - G.projection_norm(Am, Bm, f, c, r)[0]) / (2 * h)
                an = grad[e].real if part == 1.0 else grad[e].imag
                assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-3 * np.max(np.abs(grad))), (which, e, part, fd, an)


def _nearest_eig(A, B, c):
    ev = sla.eigvals(A.toarray(), None if B is None else B.toarray())
    return ev[np.argmin(np.abs(ev - c))]


@pytest.mark.parametrize("general_B", [False, True])
def test_eigenvalue_grad_against_dense_eig_and_differences(general_B):
    A, B = _small_pencil(3, general_B)
    lam0 = _nearest_eig(A, B, 30.0)
    # radius 0.1: the nearest other eigenvalue (0.92 away) leaves a quadrature error ~(0.1/0.92)^16
    lam, dA, dB = G.eigenvalue_grad(A, B, lam0, 0.1)
    assert abs(lam - lam0) <= 1e-10 * abs(lam0)
    rng = np.random.default_rng(5)
    h = 1e-5
    scale = max(np.max(np.abs(dA)), np.max(np.abs(dB)))
    for M, d, which in ((A, dA, "A"), (B, dB, "B")):
        for e in rng.choice(M.nnz, 6, replace=False):
            Ap, Bp = (_perturb(A, e, h), B) if which == "A" else (A, _perturb(B, e, h))
            Am, Bm = (_perturb(A, e, -h), B) if which == "A" else (A, _perturb(B, e, -h))
            fd = (_nearest_eig(Ap, Bp, lam0) - _nearest_eig(Am, Bm, lam0)) / (2 * h)
            # dense eig is accurate to ~1e-14 ||A||: the differences carry ~1e-9 of noise
            assert abs(fd - d[e]) <= 1e-5 * max(abs(d[e]), 1e-2 * scale) + 5e-9, (which, e, fd, d[e])
    # λ(tA, B) = t λ  and  λ(tA, tB) = λ
    assert abs(np.sum(A.data * dA) - lam) <= 1e-9 * abs(lam)
    assert abs(np.sum(A.data * dA) + np.sum(B.data * dB)) <= 1e-9 * abs(lam)


def test_eigenvalue_grad_shift_invariance_identity_B():
    A, _ = _small_pencil(4)
    lam0 = _nearest_eig(A, None, 30.0)
    lam, dA, dB = G.eigenvalue_grad(A, None, lam0, 0.1)
    assert dB is None
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    diag = rows == A.indices
    # λ(A + tI) = λ + t
    assert abs(np.sum(dA[diag]) - 1.0) <= 1e-9
    assert abs(np.sum(A.data * dA) - lam) <= 1e-9 * abs(lam)
