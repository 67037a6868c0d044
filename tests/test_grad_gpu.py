"""GPU gradients (sim_projection_norm[_grad], sim_eigenvalue_grad, and the
torch.autograd.Function wrappers) against the oracle gradients of
oracle/grad.py and against central finite differences on the GPU."""
import json
import os

import numpy as np
import pytest

from oracle import grad as G
from workloads import cdr_axes, cdr_csr, complex_gaussian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def simlib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g

    g.build()
    import paper_2006_16117_gb300 as sim

    return sim


def _pencil(general_B):
    import scipy.sparse as sp

    rng = np.random.default_rng(0)
    A = cdr_csr((7, 6), (3.0, -2.0), rng.uniform(0, 1, 42) + 0.3j * rng.uniform(-1, 1, 42)).to_scipy()
    if general_B:
        B = sp.diags([0.1 * rng.standard_normal(41), 1.5 + rng.uniform(0, 0.5, 42), 0.1 * rng.standard_normal(41)],
                     [-1, 0, 1], format="csr", dtype=np.complex128)
    else:
        B = sp.diags(rng.uniform(1, 2, 42), format="csr", dtype=np.complex128)
    return A, B


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("general_B", [False, True])
@pytest.mark.parametrize("keep", [True, False])
def test_projection_norm_grad_matches_oracle(simlib, precision, general_B, keep):
    A, B = _pencil(general_B)
    f = complex_gaussian(A.shape[0], 4)
    c, r = 40.0 + 0.2j, 25.0
    phi_o, gA_o, gB_o = G.projection_norm_grad(A, B, f, c, r)
    s = simlib.Sim((A.indptr, A.indices, A.data), (B.indptr, B.indices, B.data),
                   simlib.sim_default_options(precision=precision))
    phi = s.projection_norm(c, r, f, 16, keep)
    gA, gB = s.projection_norm_grad(A.nnz, B.nnz)
    assert abs(phi - phi_o) <= 1e-10 * phi_o
    assert _rel(gA, gA_o) <= 1e-8
    assert _rel(gB, gB_o) <= 1e-8
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("general_B", [False, True])
def test_eigenvalue_grad_matches_oracle(simlib, precision, general_B):
    import scipy.linalg as sla

    A, B = _pencil(general_B)
    ev = sla.eigvals(A.toarray(), B.toarray())
    lam0 = ev[np.argmin(np.abs(ev - 30.0))]
    lam_o, dA_o, dB_o = G.eigenvalue_grad(A, B, lam0, 0.1)
    s = simlib.Sim((A.indptr, A.indices, A.data), (B.indptr, B.indices, B.data),
                   simlib.sim_default_options(precision=precision))
    lam, dA, dB = s.eigenvalue_grad(lam0, 0.1, A.nnz, B.nnz)
    assert abs(lam - lam_o) <= 1e-10 * abs(lam_o)
    assert _rel(dA, dA_o) <= 1e-8
    assert _rel(dB, dB_o) <= 1e-8
    s.close()


def test_separable_path_gradients_match_oracle(simlib):
    dims, beta = (20, 17), (1.0, 0.5)
    rng = np.random.default_rng(3)
    A = cdr_csr(dims, beta, rng.uniform(0, 1, 340)).to_scipy()
    f = complex_gaussian(340, 6)
    c, r = 60.0 + 0.0j, 12.0
    phi_o, gA_o, _ = G.projection_norm_grad(A, None, f, c, r)
    s = simlib.Sim((A.indptr, A.indices, A.data), None, simlib.sim_default_options(precision="mixed"))
    s.set_separable(dims, cdr_axes(dims, beta))
    phi = s.projection_norm(c, r, f)
    gA, _ = s.projection_norm_grad(A.nnz)
    assert abs(phi - phi_o) <= 1e-10 * phi_o
    assert _rel(gA, gA_o) <= 1e-8
    s.close()


def test_autograd_functions_and_finite_differences(simlib):
    from paper_2006_16117_gb300 import autograd as AG

    A, B = _pencil(False)
    f = torch.from_numpy(complex_gaussian(A.shape[0], 4)).cuda()
    c, r = 40.0 + 0.2j, 25.0
    s = simlib.Sim((A.indptr, A.indices, A.data), (B.indptr, B.indices, B.data))
    a = torch.from_numpy(A.data.copy()).cuda().requires_grad_(True)
    phi = AG.projection_norm(a, s, c, r, f)
    phi.backward()
    _, gA_o, _ = G.projection_norm_grad(A, B, f.cpu().numpy(), c, r)
    assert _rel(a.grad.cpu().numpy(), gA_o) <= 1e-8
    # central differences of Φ through the same handle (values updated in place);
    # h = 1e-4 keeps the solves' rounding (~1e-12 Φ / h) below 1e-5 of the derivatives
    h = 1e-4
    rng = np.random.default_rng(1)
    base = torch.from_numpy(A.data.copy()).cuda()
    for e in rng.choice(A.nnz, 8, replace=False):
        for part in (1.0, 1j):
            ap, am = base.clone(), base.clone()
            ap[e] += h * part
            am[e] -= h * part
            fd = (AG.projection_norm(ap, s, c, r, f).item() - AG.projection_norm(am, s, c, r, f).item()) / (2 * h)
            an = gA_o[e].real if part == 1.0 else gA_o[e].imag
            assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-3 * np.max(np.abs(gA_o)))
    # the eigenvalue: backward of Re λ gives conj(dλ/da)
    import scipy.linalg as sla

    ev = sla.eigvals(A.toarray(), B.toarray())
    lam0 = ev[np.argmin(np.abs(ev - 30.0))]
    a2 = torch.from_numpy(A.data.copy()).cuda().requires_grad_(True)
    lam = AG.eigenvalue(a2, s, lam0, 0.1)
    lam.real.backward()
    _, dA_o, _ = G.eigenvalue_grad(A, B, lam0, 0.1)
    assert _rel(a2.grad.cpu().numpy(), np.conj(dA_o)) <= 1e-8
    s.close()


def test_cdr2d_full_size_gradients_match_oracle_record_and_differences(simlib):
    """n = 250,000, separable preconditioner, mixed precision: Φ, λ and their
    gradients on 32 reaction coefficients equal the oracle's (recorded by
    tests/golden/make_cdr2d_grad_record.py) and central differences (h = 1e-6)."""
    from workloads.configs import config_cdr2d

    with open(os.path.join(os.path.dirname(__file__), "golden", "cdr2d500_grad_record.json")) as fh:
        ref = json.load(fh)
    w = config_cdr2d(500)
    A = w.A
    c = complex(*ref["center"])
    r = ref["radius"]
    pos = np.array(ref["positions"])
    s = simlib.Sim(A, None, simlib.sim_default_options(precision="mixed"))
    s.set_separable(*w.separable)
    phi = s.projection_norm(c, r, w.f)
    gA, _ = s.projection_norm_grad(A.nnz)
    g_ref = np.array(ref["grad_phi_re"]) + 1j * np.array(ref["grad_phi_im"])
    assert abs(phi - ref["phi"]) <= 1e-9 * ref["phi"]
    assert _rel(gA[pos], g_ref) <= 1e-7
    lam, dA, _ = s.eigenvalue_grad(c, r, A.nnz)
    d_ref = np.array(ref["dlam_re"]) + 1j * np.array(ref["dlam_im"])
    assert abs(lam - complex(*ref["lam"])) <= 1e-10 * abs(lam)
    assert _rel(dA[pos], d_ref) <= 1e-7
    s.close()
    # central differences (h = 1e-6) on the GPU, FP64 solves to 1e-14 so that
    # the differences' rounding (~tol·Φ/h) stays below 1e-5 of them, along 32 random directions of
    # the reaction coefficients: every diagonal entry at once, with the sign of
    # its gradient and a random size in [0.5, 1.5] (one coefficient alone moves
    # Φ by ~1e-12 relative, the rounding level of the solves)
    M = A.to_scipy()
    rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    diag = np.nonzero(rows == M.indices)[0]
    vals = A.data.copy()
    h = 1e-6
    rng = np.random.default_rng(11)
    s = simlib.Sim(A, None, simlib.sim_default_options(precision="fp64", inner_tol=1e-14, inner_max_iter=200))
    s.set_separable(*w.separable)
    for _ in range(32):
        v = np.sign(gA[diag].real) * rng.uniform(0.5, 1.5, diag.size)
        vp, vm = vals.copy(), vals.copy()
        vp[diag] += h * v
        vm[diag] -= h * v
        s.update_values(vp)
        fp = s.projection_norm(c, r, w.f, keep=False)
        s.update_values(vm)
        fm = s.projection_norm(c, r, w.f, keep=False)
        fd = (fp - fm) / (2 * h)
        an = float(np.dot(gA[diag].real, v))
        assert abs(fd - an) <= 1e-5 * abs(an) + 2e-6 * phi, (fd, an)
    s.close()
