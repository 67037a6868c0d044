"""Pins for the CPU oracle: each check compares it with something other than
itself — closed forms, invariants, dense library eigensolvers, brute force —
so that a dropped term, a wrong sign or index or a transposed operand in the
oracle fails at least one of them."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import simm as S
from oracle.inertia import count_below
from oracle.philox import philox4x64, random_vectors
from workloads import (
    block_diag_csr,
    cd2d_csr,
    cd2d_eigenvalues,
    config_jordan_small,
    dense_to_csr,
    diag_csr,
    jordan_csr,
    pair_blocks_csr,
    tridiag_toeplitz_csr,
)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _closed_form_indicator(lam, f, c, s):
    """Ĩ for a diagonal matrix (B = I) by the N-point trapezoid identity
    (1/N) Σ_j ω^j/(ω^j - u) = 1/(1 - u^N) (u = (λ - c)/r, ω = e^{2πi/N}):
    component k of Σ_j w_j (A - z_j)^{-1} f is -f_k/(1 - u_k^N)."""
    r = s / math.sqrt(2.0)
    u = (lam - c) / r
    n8 = np.linalg.norm(f / (1 - u**8))
    n4 = np.linalg.norm(f / (1 - u**4))
    return n8 / n4


def test_trapezoid_identity_numerically():
    # the identity the closed form rests on, checked by direct summation
    for N in (4, 8, 16):
        w = np.exp(2j * np.pi * np.arange(N) / N)
        for u in (0.3 + 0.1j, 1.7 - 0.4j, -0.9j):
            lhs = np.mean(w / (w - u))
            assert abs(lhs - 1 / (1 - u**N)) < 1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_indicator_closed_form_diagonal(seed):
    rng = np.random.default_rng(seed)
    n = 30  # n < m: the Krylov space is exact
    lam = rng.uniform(-3, 3, n) + 1j * rng.uniform(-3, 3, n)
    A = sp.diags(lam).tocsr()
    B = sp.identity(n, format="csr", dtype=complex)
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ks = S.cayley_arnoldi(A, B, 0.37 + 0.21j, f, 50)
    assert ks.m_eff == n
    centers = np.array([0.1 + 0.2j, -1.3 + 0.7j, 2.2 - 2.1j, 0.0 + 0.0j])
    sides = np.array([0.5, 1.0, 0.25, 6.0])
    ind, rho = S.evaluate_squares(ks, centers, sides)
    for q in range(centers.size):
        ref = _closed_form_indicator(lam, f, centers[q], sides[q])
        assert abs(ind[q] - ref) <= 1e-9 * max(1.0, ref), (q, ind[q], ref)
    assert np.all(rho < 1e-10)  # exact Krylov space: h_{m+1,m} = 0


def test_single_eigenvalue_indicator_and_paper_threshold_example():
    # one eigenvalue at u = (λ - c)/r: Ĩ = |1 - u^4| / |1 - u^8| = 1/|1 + u^4|
    n0, C, printed, delta0 = np.loadtxt(os.path.join(GOLDEN, "threshold_example.txt"))
    A = sp.csr_matrix(np.array([[0.0 + 0j]]))
    B = sp.identity(1, format="csr", dtype=complex)
    s = 1.0
    r = s / math.sqrt(2)
    u = math.e ** C  # an outside eigenvalue with |u| = e^C (exponent C per node)
    c = -u * r + 0j  # put λ = 0 at c + u r
    ks = S.cayley_arnoldi(A, B, 0.4 + 0.3j, np.array([1.0 + 0j]), 50)
    ind, _ = S.evaluate_squares(ks, np.array([c]), np.array([s]))
    assert abs(ind[0] - 1 / abs(1 + u**4)) < 1e-12
    assert round(ind[0], 3) == printed  # Sec. 3.1: ~0.018 for n0 = 4, C = 1
    assert ind[0] < delta0
    # inside the circle the indicator stays near 1: >= 1/2 for |u| < 1
    for uu in (0.0, 0.5, 0.9j, -0.7 + 0.2j):
        ks2 = S.cayley_arnoldi(A, B, 3.0 + 1j, np.array([1.0 + 0j]), 50)
        ind2, _ = S.evaluate_squares(ks2, np.array([-uu * r]), np.array([s]))
        assert abs(ind2[0] - 1 / abs(1 + uu**4)) < 1e-12
        assert ind2[0] >= 0.5


def test_exact_krylov_matches_dense_resolvent_nonnormal():
    rng = np.random.default_rng(5)
    n = 40
    Ad = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Ad = np.triu(Ad, -2)  # non-normal, banded-ish
    Bd = np.eye(n) + 0.1 * np.diag(rng.uniform(0, 1, n))
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    A, B = sp.csr_matrix(Ad), sp.csr_matrix(Bd)
    sigma = 0.3 + 0.2j
    ks = S.cayley_arnoldi(A, B, sigma, f, 50)
    c, s = 0.5 - 0.4j, 2.0
    off = S.node_offsets(np.array(s))
    z = c + off
    xs = np.array([np.linalg.solve(Ad - zj * Bd, f) for zj in z])
    Y8 = (off / 8) @ xs
    Y4 = (off[0::2] / 4) @ xs[0::2]
    ref = np.linalg.norm(Y8) / np.linalg.norm(Y4)
    ind, _ = S.evaluate_squares(ks, np.array([c]), np.array([s]))
    assert abs(ind[0] - ref) < 1e-9 * ref


def test_arnoldi_relation_and_orthonormality():
    w = cd2d_csr(10, (1.0, 0.5))
    A = w.to_scipy()
    n = A.shape[0]
    B = sp.diags(np.linspace(1, 2, n)).tocsr().astype(complex)
    f = np.random.default_rng(2).standard_normal(n) + 0j
    sigma = 250.0 + 0.3j
    m = 30
    ks = S.cayley_arnoldi(A, B, sigma, f, m, keep_basis=True)
    M = np.linalg.solve((A - sigma * B).toarray(), B.toarray())
    V = ks.V
    Hm = ks.H[:m, :m]
    rel = M @ V[:, :m] - V[:, :m] @ Hm - np.outer(V[:, m], ks.H[m, m - 1] * np.eye(m)[m - 1])
    assert np.linalg.norm(rel) / np.linalg.norm(Hm) < 1e-12
    assert np.linalg.norm(V.conj().T @ V - np.eye(m + 1)) < 1e-12
    b = np.linalg.solve((A - sigma * B).toarray(), f)
    assert abs(ks.beta - np.linalg.norm(b)) < 1e-12 * ks.beta
    assert np.linalg.norm(V[:, 0] * ks.beta - b) < 1e-10 * ks.beta
    # Hessenberg structure: zeros below the first subdiagonal, real positive subdiagonal
    assert np.all(np.abs(np.tril(ks.H, -2)) == 0)
    sub = np.diag(ks.H, -1)
    assert np.all(sub.real > 0) and np.all(sub.imag == 0)


def test_residual_formula_equals_explicit_residual():
    w = cd2d_csr(9, (1.0, 0.5))
    A = w.to_scipy()
    n = A.shape[0]
    B = sp.identity(n, format="csr", dtype=complex)
    f = np.random.default_rng(4).standard_normal(n) + 1j
    sigma = 300.0 + 0.5j
    m = 20
    ks = S.cayley_arnoldi(A, B, sigma, f, m, keep_basis=True)
    M = np.linalg.solve((A - sigma * B).toarray(), B.toarray())
    b = ks.V[:, 0] * ks.beta
    z = np.array([301.0 + 0.1j, 420.0 - 2j, 150.0 + 3j, 600.0 + 1j])
    y, rho = S.projected_solve(ks, z)
    assert rho.max() > 1e-6  # far points: the 20-dimensional space is not exact
    for q, zq in enumerate(z):
        x = ks.V[:, :m] @ y[q]
        r = b - (x + (sigma - zq) * (M @ x))
        explicit = np.linalg.norm(r) / np.linalg.norm(y[q])
        assert abs(explicit - rho[q]) <= 1e-7 * explicit + 1e-12
        # the Galerkin system itself: (I + (σ - z)H) y = β e1
        T = np.eye(m) + (sigma - zq) * ks.H[:m, :m]
        e = np.zeros(m, complex)
        e[0] = ks.beta
        assert np.linalg.norm(T @ y[q] - e) < 1e-10 * ks.beta
    # the other reading of the test (option residual_scale = "beta"): the same
    # solve, the explicit residual relative to the right-hand side's norm β
    yb, rho_b = S.projected_solve(ks, z, "beta")
    assert np.array_equal(yb, y)
    for q, zq in enumerate(z):
        x = ks.V[:, :m] @ y[q]
        r = b - (x + (sigma - zq) * (M @ x))
        explicit = np.linalg.norm(r) / np.linalg.norm(b)
        assert abs(explicit - rho_b[q]) <= 1e-7 * explicit + 1e-12


def test_tiling_and_levels():
    ix, iy = S.initial_tiling((0.0, 3.5, -1.0, 0.0), 1.0)
    assert list(ix) == [0, 1, 2, 3] and list(iy) == [0, 0, 0, 0]
    ix, iy = S.initial_tiling((0.0, 2.0, 0.0, 2.0), 1.0)
    assert list(zip(iy, ix)) == [(0, 0), (0, 1), (1, 0), (1, 1)]
    assert S.num_levels(1.0, 1e-6) == 21
    assert 1.0 / 2 ** (S.num_levels(1.0, 1e-6) - 1) <= 1e-6 < 1.0 / 2 ** (S.num_levels(1.0, 1e-6) - 2)
    off = S.node_offsets(np.array(2.0))
    # odd nodes are the square's corners; even nodes lie at radius s/sqrt(2)
    assert np.allclose(off[1::2], [1 + 1j, -1 + 1j, -1 - 1j, 1 - 1j])
    assert np.allclose(np.abs(off), math.sqrt(2.0))
    assert np.allclose(np.angle(off), np.angle(np.exp(2j * np.pi * np.arange(8) / 8)))


def _match(est, ref, tol):
    """Greedy one-to-one match of estimates to reference eigenvalues."""
    est = np.asarray(est)
    ref = np.asarray(ref)
    used = np.zeros(ref.size, bool)
    worst = 0.0
    for e in est:
        d = np.abs(ref - e)
        d[used] = np.inf
        j = int(np.argmin(d))
        used[j] = True
        worst = max(worst, d[j])
    return worst


def test_end_to_end_small_convection_diffusion(small_workload):
    w = small_workload
    res = S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))
    assert res.eigenvalues.size == w.expected_count == 50
    assert _match(res.eigenvalues, w.reference_eigs, 1.0) <= w.options["h0"]
    assert np.all(res.multiplicities == 1)


def test_tridiagonal_toeplitz_complex_segment():
    n = 60
    a, b, c = 2.0 + 1.0j, 1.0 + 0.5j, 0.6 - 0.2j
    A = tridiag_toeplitz_csr(n, b, a, c).to_scipy()
    k = np.arange(1, n + 1)
    lam = a + 2 * np.sqrt(b * c) * np.cos(k * np.pi / (n + 1))
    # region around a part of the segment, edges between eigenvalues along Re
    lr = np.sort(lam.real)
    lo, hi = 0.5 * (lr[19] + lr[20]), 0.5 * (lr[29] + lr[30])
    im = lam.imag
    region = (lo, hi, im.min() - 0.11, im.max() + 0.13)
    inside = lam[(lam.real > lo) & (lam.real < hi)]
    f = np.random.default_rng(7).standard_normal(n) + 0j
    res = S.sim_m(A, None, region, f, S.Options(h0=1e-6, init_side=0.25))
    assert res.eigenvalues.size == inside.size
    assert _match(res.eigenvalues, inside, 1.0) <= 1e-6


def test_complex_pairs():
    al = np.array([1.0, 1.5, 2.0, 2.5])
    be = np.array([0.3, -0.2, 0.45, 0.1])
    A = pair_blocks_csr(al, be).to_scipy()
    lam = np.concatenate([al + 1j * be, al - 1j * be])
    region = (1.2, 2.3, -0.6, 0.6)
    inside = lam[(lam.real > 1.2) & (lam.real < 2.3)]
    f = np.random.default_rng(8).standard_normal(A.shape[0]) + 0.5j
    res = S.sim_m(A, None, region, f, S.Options(h0=1e-6, init_side=0.3))
    assert res.eigenvalues.size == inside.size == 4
    assert _match(res.eigenvalues, inside, 1.0) <= 1e-6
    assert np.all(res.multiplicities == 1)


def test_generalized_pencil_vs_dense_qz():
    N = 15
    A0 = cd2d_csr(N, (1.0, 0.5))
    bd = np.random.default_rng(11).uniform(1.0, 2.0, A0.n)
    A, B = A0.to_scipy(), diag_csr(bd).to_scipy()
    lam = sla.eigvals(A.toarray(), B.toarray())
    lr = np.sort(lam.real)
    lo, hi = 0.5 * (lr[99] + lr[100]), 0.5 * (lr[119] + lr[120])
    inside = lam[(lam.real > lo) & (lam.real < hi)]
    assert inside.size == 20
    f = np.random.default_rng(12).standard_normal(A0.n) + 0j
    res = S.sim_m(A, B, (lo, hi, -0.3, 0.7), f, S.Options(h0=1e-6))
    assert res.eigenvalues.size == 20
    assert _match(res.eigenvalues, inside, 1.0) <= 1e-6
    # and inertia counts the same number of eigenvalues in [lo, hi]
    assert count_below(N, (1.0, 0.5), bd, hi) - count_below(N, (1.0, 0.5), bd, lo) == 20


def _generalized_case():
    N = 15
    A0 = cd2d_csr(N, (1.0, 0.5))
    bd = np.random.default_rng(11).uniform(1.0, 2.0, A0.n)
    A, B = A0.to_scipy(), diag_csr(bd).to_scipy()
    lam = sla.eigvals(A.toarray(), B.toarray())
    lr = np.sort(lam.real)
    lo, hi = 0.5 * (lr[99] + lr[100]), 0.5 * (lr[119] + lr[120])
    f = np.random.default_rng(12).standard_normal(A0.n) + 0j
    return A0, bd, A, B, lam[(lam.real > lo) & (lam.real < hi)], (lo, hi, -0.3, 0.7), f


def test_refinement_and_projection_on_generalized_pencil():
    # B ≠ I: the refined values σ + 1/d against dense QZ, and P f against A x = λ B x.
    _, _, A, B, inside, region, f = _generalized_case()
    sim = S.SimM(A, B, S.Options(h0=1e-6))
    sim.set_region(region, f)
    sim.solve_levels()
    sim.merge()
    ref, flag = sim.refine()
    assert flag.all() and ref.size == inside.size == 20
    assert _match(ref, inside, 1.0) <= 1e-8
    Ad, Bd = A.toarray(), B.toarray()
    for c in (0, 9, 19):
        x = sim.projection(c)
        assert np.linalg.norm(Ad @ x - ref[c] * (Bd @ x)) <= 1e-8 * abs(ref[c]) * np.linalg.norm(Bd @ x)


def test_ritz_refinement_beats_h0_on_closed_form(small_workload):
    # Sec. 3.2: λ = σ + 1/d over the eigenvalues d of H_m.  Against the closed
    # form, every refined eigenvalue of the 50-eigenvalue case is far inside h0
    # and closer than the square-centroid estimate it replaces.
    w = small_workload
    sim = S.SimM(w.A.to_scipy(), None, S.Options(**w.options))
    sim.set_region(w.region, w.f)
    sim.solve_levels()
    sim.merge()
    est = sim.clusters["estimate"]
    ref, flag = sim.refine()
    truth = np.sort_complex(w.reference_eigs)
    err_est = np.min(np.abs(est[:, None] - truth[None, :]), axis=1)
    err_ref = np.min(np.abs(ref[:, None] - truth[None, :]), axis=1)
    assert flag.all()
    assert err_ref.max() <= 1e-8
    assert np.all(err_ref <= err_est)
    # the nearest-Ritz-value rule picks the eigenvalue the estimate belongs to
    assert np.array_equal(np.argmin(np.abs(ref[:, None] - truth[None, :]), axis=1),
                          np.argmin(np.abs(est[:, None] - truth[None, :]), axis=1))


def test_projection_is_an_eigenvector(small_workload):
    # Remark 3.5: for a simple eigenvalue, P f on the cluster's circle is a right
    # eigenvector.  Checked against dense eig: residual and angle at rounding level.
    w = small_workload
    A = w.A.to_scipy()
    sim = S.SimM(A, None, S.Options(**w.options))
    sim.set_region(w.region, w.f)
    sim.solve_levels()
    sim.merge()
    ref, _ = sim.refine()
    lam_d, X = np.linalg.eig(A.toarray())
    for c in (0, 17, 49):
        x = sim.projection(c)
        assert np.linalg.norm(A @ x - ref[c] * x) <= 1e-10 * abs(ref[c]) * np.linalg.norm(x)
        v = X[:, int(np.argmin(np.abs(lam_d - ref[c])))]
        assert abs(np.vdot(v, x)) >= (1 - 1e-10) * np.linalg.norm(v) * np.linalg.norm(x)


def test_jordan_multiplicity():
    w = config_jordan_small()
    res = S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))
    assert res.eigenvalues.size == w.reference_eigs.size
    assert np.array_equal(res.multiplicities, w.reference_mult)
    assert int(res.multiplicities.sum()) == w.expected_count
    simple = w.reference_mult == 1
    assert _match(res.eigenvalues[simple], w.reference_eigs[simple], 1.0) <= 1e-6
    # defective eigenvalues: located as one cluster of algebraic multiplicity 4
    assert _match(res.eigenvalues[~simple], w.reference_eigs[~simple], 1.0) <= 1e-6


def test_laplacian_degenerate_multiplicities_vs_dense():
    N = 8
    A = cd2d_csr(N, (0.0, 0.0)).to_scipy()
    ev = np.sort(np.linalg.eigvalsh(A.toarray().real))
    # group the dense spectrum into clusters (exact degeneracies of μ_k + μ_l)
    groups = []
    for x in ev:
        if groups and abs(x - groups[-1][0]) < 1e-7 * max(1.0, abs(x)):
            groups[-1][1] += 1
        else:
            groups.append([x, 1])
    h = 1.0 / (N + 1)
    centre = 4.0 / h**2  # k + l = N + 1: multiplicity N
    vals = np.array([g[0] for g in groups])
    mults = np.array([g[1] for g in groups])
    j = int(np.argmin(np.abs(vals - centre)))
    assert mults[j] == N
    lo, hi = 0.5 * (vals[j - 3] + vals[j - 2]), 0.5 * (vals[j + 2] + vals[j + 3])
    sel = (vals > lo) & (vals < hi)
    f = np.random.default_rng(13).standard_normal(A.shape[0]) + 0j
    res = S.sim_m(A, None, (lo, hi, -0.4, 0.6), f, S.Options(h0=1e-6))
    assert res.eigenvalues.size == int(sel.sum())
    assert _match(res.eigenvalues, vals[sel], 1.0) <= 1e-6
    order = np.argsort(vals[sel])
    assert np.array_equal(res.multiplicities, mults[sel][order])


def test_identity_B_equals_standard_problem(small_workload):
    w = small_workload
    A = w.A.to_scipy()
    ks1 = S.cayley_arnoldi(A, sp.identity(A.shape[0], format="csr", dtype=complex), 4000 + 0.2j, w.f, 20)
    ks2 = S.cayley_arnoldi(A, sp.csr_matrix(np.eye(A.shape[0], dtype=complex)), 4000 + 0.2j, w.f, 20)
    assert np.allclose(ks1.H, ks2.H, atol=1e-12)
    # standard problem: b = (A - σI)^{-1} f
    b = np.linalg.solve(A.toarray() - (4000 + 0.2j) * np.eye(A.shape[0]), w.f)
    assert abs(ks1.beta - np.linalg.norm(b)) < 1e-12 * ks1.beta


def test_philox_matches_numpy_and_known_answer():
    # numpy's Philox (4x64, 10 rounds) emits counter+1 first
    key = (0x1234567890ABCDEF, 0x0FEDCBA987654321)
    bg = np.random.Philox(key=list(key), counter=[0, 0, 0, 0])
    raw = bg.random_raw(8)
    for c in range(2):
        out = philox4x64([np.uint64(c + 1), np.uint64(0), np.uint64(0), np.uint64(0)],
                         [np.uint64(key[0]), np.uint64(key[1])])
        assert [int(v) for v in out] == [int(v) for v in raw[4 * c: 4 * c + 4]]
    # Random123 known answer for counter = key = 0
    out = philox4x64([np.uint64(0)] * 4, [np.uint64(0)] * 2)
    assert [int(v) for v in out] == [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC,
                                    0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]
    F = random_vectors(7, 20000, 3)
    assert F.shape == (20000, 3)
    assert abs(F.mean()) < 0.03
    assert abs(np.mean(np.abs(F) ** 2) - 1.0) < 0.03
    assert np.array_equal(random_vectors(7, 50, 2, first=1)[:, 0], F[:50, 1])


def test_inertia_counts_vs_dense():
    N = 10
    bd = np.random.default_rng(21).uniform(1, 2, N * N)
    A = cd2d_csr(N, (1.0, 0.5)).to_dense()
    ev = np.sort(np.linalg.eigvals(A / bd[:, None]).real)
    for x in np.linspace(ev[0] - 1, ev[-1] + 1, 13):
        assert count_below(N, (1.0, 0.5), bd, x) == int(np.sum(ev < x))


def test_closed_form_cd_spectrum_vs_dense():
    N = 12
    A = cd2d_csr(N, (1.0, 0.5)).to_dense()
    ev = np.linalg.eigvals(A)
    ref = cd2d_eigenvalues(N, (1.0, 0.5))
    assert np.max(np.abs(np.sort(ev.real) - np.sort(ref.real))) < 1e-9 * np.abs(ref).max()
    assert np.max(np.abs(ev.imag)) < 1e-8 * np.abs(ref).max()


# -- planted mistakes: each must make a pin fail -------------------------------
def test_planted_mistakes_are_caught(monkeypatch):
    rng = np.random.default_rng(0)
    n = 12
    lam = rng.uniform(-2, 2, n) + 1j * rng.uniform(-2, 2, n)
    A = sp.diags(lam).tocsr()
    B = sp.identity(n, format="csr", dtype=complex)
    f = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ks = S.cayley_arnoldi(A, B, 0.1 + 0.1j, f, 50)
    c, s = 0.2 + 0.1j, 1.5
    ref = _closed_form_indicator(lam, f, c, s)
    good, _ = S.evaluate_squares(ks, np.array([c]), np.array([s]))
    assert abs(good[0] - ref) < 1e-9 * ref
    real_off = S.node_offsets
    # (1) a wrong sign on one node
    monkeypatch.setattr(S, "node_offsets", lambda s_: real_off(s_) * np.array([1, 1, -1, 1, 1, 1, 1, 1]))
    bad, _ = S.evaluate_squares(ks, np.array([c]), np.array([s]))
    assert abs(bad[0] - ref) > 1e-6 * ref
    monkeypatch.setattr(S, "node_offsets", real_off)
    # (2) a transposed Hessenberg (non-normal pencil: the dense resolvent is the reference)
    rng2 = np.random.default_rng(5)
    Ad = np.triu(rng2.standard_normal((30, 30)) + 1j * rng2.standard_normal((30, 30)), -2)
    f2 = rng2.standard_normal(30) + 0j
    ks2 = S.cayley_arnoldi(sp.csr_matrix(Ad), sp.identity(30, format="csr", dtype=complex), 0.3 + 0.2j, f2, 50)
    c2, s2 = 0.5 - 0.4j, 2.0
    off2 = S.node_offsets(np.array(s2))
    xs = np.array([np.linalg.solve(Ad - zj * np.eye(30), f2) for zj in c2 + off2])
    ref2 = np.linalg.norm((off2 / 8) @ xs) / np.linalg.norm((off2[0::2] / 4) @ xs[0::2])
    ok2, _ = S.evaluate_squares(ks2, np.array([c2]), np.array([s2]))
    assert abs(ok2[0] - ref2) < 1e-9 * ref2
    ks_t = S.KrylovSpace(ks2.sigma, np.vstack([ks2.H[:-1].T, ks2.H[-1:]]), ks2.beta, ks2.m_eff)
    bad, _ = S.evaluate_squares(ks_t, np.array([c2]), np.array([s2]))
    assert abs(bad[0] - ref2) > 1e-6 * ref2
    # (3) σ - z replaced by z - σ in the projected system: (I + (z - σ)H) y = βe1
    ks_s = S.KrylovSpace(ks.sigma, -ks.H, ks.beta, ks.m_eff)
    bad, _ = S.evaluate_squares(ks_s, np.array([c]), np.array([s]))
    assert abs(bad[0] - ref) > 1e-6 * ref
    # (4) fine-rule weights without the (z_j - c) factor
    real_ind = S.indicator_from_y
    monkeypatch.setattr(S, "indicator_from_y", lambda y, off: real_ind(y, np.abs(off)))
    bad, _ = S.evaluate_squares(ks, np.array([c]), np.array([s]))
    assert abs(bad[0] - ref) > 1e-6 * ref


def test_eig_decomposition_screen_equals_direct_solve():
    """Sec. 3.2: e_m^T y = β r_m Λ c_1 equals the last entry of the direct
    Hessenberg solve for a diagonalisable, well-conditioned H_m (the Krylov
    space of a normal matrix), and its β-relative residual equals Eq. eq:error's."""
    rng = np.random.default_rng(12)
    lam = rng.uniform(0, 10, 80) + 1j * rng.uniform(-1, 1, 80)
    A = diag_csr(lam).to_scipy()
    f = rng.standard_normal(80) + 1j * rng.standard_normal(80)
    ks = S.cayley_arnoldi(A, sp.identity(80, dtype=complex, format="csr"), 5.0 + 0.3j, f, 50)
    d, P, c1, rm = S.eig_decomposition(ks)
    assert np.linalg.cond(P) < 1e6
    z = 5.0 + 0.3j + rng.uniform(-3, 3, 64) + 1j * rng.uniform(-1, 1, 64)
    y, rho_direct = S.projected_solve(ks, z, "beta")
    ym, rho_screen = S.screened_last_entry(ks, z, (d, P, c1, rm))
    # agreement to rounding of the sum: relative where e_m^T y is not tiny, and
    # within 1e-12 of the sum of the magnitudes of its terms everywhere
    alpha = ks.sigma - z
    scale = ks.beta * np.sum(np.abs(rm * c1 / (1.0 + alpha[:, None] * d)), axis=-1)
    assert np.all(np.abs(ym - y[:, -1]) <= 1e-9 * np.abs(y[:, -1]) + 1e-12 * scale)
    big = np.abs(y[:, -1]) > 1e-6 * scale
    assert big.sum() >= 10
    assert np.max(np.abs(rho_screen[big] - rho_direct[big]) / rho_direct[big]) <= 1e-9
    # and the decomposition reproduces H_m
    m = ks.m_eff
    assert np.linalg.norm(P @ np.diag(d) @ np.linalg.inv(P) - ks.H[:m, :m]) <= 1e-9 * np.linalg.norm(ks.H[:m, :m])


def test_schur_form_evaluation_equals_direct_solve():
    """The identities the levels' Schur path uses (Sec. 3.2 with the unitary
    H_m = Z T Z^H in place of P D P^{-1}), on a non-normal pencil's Krylov
    space: x = (I + αT)^{-1} β Z^H e_1 gives ||x|| = ||y||, z_m^T x = e_m^T y, and
    the indicator and residuals of whole squares equal the oracle's direct
    evaluation (scipy's complex Schur form serves as the library step)."""
    import scipy.linalg as sla

    from workloads import cd2d_csr

    A = cd2d_csr(20, (1.0, 0.5)).to_scipy()
    n = A.shape[0]
    f = np.random.default_rng(9).standard_normal(n) + 1j * np.random.default_rng(10).standard_normal(n)
    sigma = 400.0 + 0.2j
    ks = S.cayley_arnoldi(A, sp.identity(n, dtype=complex, format="csr"), sigma, f, 20)
    m = ks.m_eff
    H = ks.H[:m, :m]
    T, Z = sla.schur(H, output="complex")
    assert np.linalg.norm(Z @ T @ Z.conj().T - H) <= 1e-12 * np.linalg.norm(H)
    c = ks.beta * Z[0, :].conj()
    rng = np.random.default_rng(11)
    centers = sigma + rng.uniform(-300, 300, 12) + 1j * rng.uniform(-1, 1, 12)
    sides = rng.uniform(0.05, 2.0, 12)
    ind_direct, rmax_direct = S.evaluate_squares(ks, centers, sides)
    hlast = abs(ks.H[m, m - 1])
    for q in range(centers.size):
        off = S.node_offsets(np.array(sides[q]))
        z = centers[q] + off
        y, _ = S.projected_solve(ks, z)
        xs = []
        rho = []
        for j in range(8):
            alpha = sigma - z[j]
            x = sla.solve_triangular(np.eye(m) + alpha * T, c)
            assert abs(np.linalg.norm(x) - np.linalg.norm(y[j])) <= 1e-9 * np.linalg.norm(y[j])
            last = Z[m - 1, :] @ x
            assert abs(last - y[j][m - 1]) <= 1e-9 * np.linalg.norm(y[j])
            rho.append(abs(alpha) * hlast * abs(last) / np.linalg.norm(x))
            xs.append(x)
        xs = np.array(xs)
        s8 = np.linalg.norm(np.sum((off / 8.0)[:, None] * xs, axis=0))
        s4 = np.linalg.norm(np.sum((off[0::2] / 4.0)[:, None] * xs[0::2], axis=0))
        assert abs(s8 / s4 - ind_direct[q]) <= 1e-8 * max(1.0, ind_direct[q])
        # residuals agree to rounding (an absolute floor far below ε = 1e-8)
        assert abs(max(rho) - rmax_direct[q]) <= 1e-6 * rmax_direct[q] + 1e-13
    assert np.max(rmax_direct) > 1e-6  # the 20-dimensional space is not exact for every square
