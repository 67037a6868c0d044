"""Separable principal part: the fast-diagonalisation preconditioner of the
inner solves (sim_set_separable) and the convection–diffusion–reaction
workloads it serves (2-D with a real reaction, 3-D with a complex one).

CPU: the workload generators against closed forms and the oracle against
dense eigensolvers and Weyl's bound.  GPU: shifted solves against sparse LU,
and whole SIM-M runs equal to the oracle's."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import simm as S
from workloads import cdr_csr, cdr_separable_eigenvalues, complex_gaussian
from workloads.configs import config_cdr2d, config_cdr3d


def test_cdr_generator_matches_closed_form_spectrum():
    for dims, beta in (((6, 5), (1.0, 0.5)), ((4, 5, 3), (1.0, 0.5, 0.25))):
        A = cdr_csr(dims, beta).to_scipy().toarray()
        ev = np.sort(np.linalg.eigvals(A).real)
        ref = np.sort(cdr_separable_eigenvalues(dims, beta).real)
        assert np.max(np.abs(ev - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_oracle_cdr2d_low_end_against_weyl_bound():
    """Real reaction 0 <= c <= 1 on a matrix similar to a symmetric one: every
    eigenvalue is real and within [0, 1] above a separable eigenvalue, so the
    region's count is the closed-form one."""
    w = config_cdr2d(30, 8)
    r = S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))
    assert r.eigenvalues.size == w.expected_count
    assert np.array_equal(r.multiplicities, np.ones(w.expected_count, dtype=np.int64))
    assert np.max(np.abs(r.eigenvalues.imag)) <= 1e-6
    dense = np.sort(np.linalg.eigvals(w.A.to_scipy().toarray()).real)[: w.expected_count]
    assert np.max(np.abs(np.sort(r.eigenvalues.real) - dense)) <= 1e-6
    sep = np.sort(cdr_separable_eigenvalues((30, 30), (1.0, 0.5)).real)[: w.expected_count]
    assert np.all((dense >= sep - 1e-9) & (dense <= sep + 1.0 + 1e-9))


@pytest.fixture(scope="module")
def cdr3d_small():
    w = config_cdr3d(12, 30.0)
    ref = S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))
    return w, ref


def test_oracle_cdr3d_against_dense_eig(cdr3d_small):
    w, ref = cdr3d_small
    ev = np.linalg.eigvals(w.A.to_scipy().toarray())
    lo, hi, ilo, ihi = w.region
    inside = ev[(ev.real >= lo) & (ev.real <= hi) & (ev.imag >= ilo) & (ev.imag <= ihi)]
    inside = inside[np.lexsort((inside.imag, inside.real))]
    assert ref.eigenvalues.size == inside.size >= 20
    assert np.max(np.abs(ref.eigenvalues - inside)) <= 1e-6
    assert np.array_equal(ref.multiplicities, np.ones(inside.size, dtype=np.int64))


# ---------------------------------------------------------------------------
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def simlib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g

    g.build()
    import paper_2006_16117_gb300 as sim

    return sim


def _separable_sim(simlib, A, dims, axes, precision, B=None):
    s = simlib.Sim(A, B, simlib.sim_default_options(precision=precision))
    s.set_separable(dims, axes)
    return s


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["cd2d", "cdr3d", "cd2d_scaled_B"])
def test_separable_shifted_solve_matches_sparse_lu(simlib, precision, case):
    from workloads import cdr_axes, diag_csr

    rng = np.random.default_rng(21)
    if case == "cdr3d":
        dims, beta = (10, 12, 9), (1.0, 0.5, 0.25)
        react = np.sqrt(rng.uniform(size=np.prod(dims))) * np.exp(2j * np.pi * rng.uniform(size=np.prod(dims)))
        sigma = 700.0 + 0.2j
    else:
        dims, beta, react, sigma = (40, 33), (1.0, 0.5), None, 3000.0 + 0.2j
    A = cdr_csr(dims, beta, react)
    n = A.n
    B = diag_csr(np.full(n, 2.0 + 0.0j)) if case == "cd2d_scaled_B" else None
    s = _separable_sim(simlib, A, dims, cdr_axes(dims, beta), precision, B)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, iters, rel = s.shifted_solve(sigma, torch.from_numpy(r).cuda())
    Bs = sp.identity(n) if B is None else B.to_scipy()
    ref = spla.splu((A.to_scipy() - sigma * Bs).tocsc()).solve(r)
    assert rel <= 1e-12
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
    if case != "cdr3d":
        assert iters <= (2 if precision == "fp64" else 4)  # exact preconditioner: one step + rounding
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("dims", [(40, 33), (10, 12, 9), (300, 7)])
def test_separable_tensor_core_mode_products_equal_cuda_cores(simlib, dims):
    """Mixed precision: the mode products on the tensor cores (TF32 with hi/lo
    splitting) and on the CUDA cores (FP32) are the same preconditioner to FP32
    accuracy, so the FP64 FGMRES around them takes the same number of steps
    (give or take one) to the same solution.  Axis lengths cover one output tile
    (33, 40), several (300) and lengths that are not multiples of 4 or 16."""
    from workloads import cdr_axes

    beta = (1.0, 0.5, 0.25)[: len(dims)]
    rng = np.random.default_rng(5)
    n = int(np.prod(dims))
    react = 0.3 * np.sqrt(rng.uniform(size=n)) * np.exp(2j * np.pi * rng.uniform(size=n))
    A = cdr_csr(dims, beta, react)
    lam = np.sort(cdr_separable_eigenvalues(dims, beta).real)
    sigma = lam[len(lam) // 3] + 0.37 + 0.2j
    r = torch.from_numpy(rng.standard_normal(n) + 1j * rng.standard_normal(n)).cuda()
    ref = spla.splu((A.to_scipy() - sigma * sp.identity(n)).tocsc()).solve(r.cpu().numpy())
    out = []
    for tc in (0, 1):
        s = simlib.Sim(A, None, simlib.sim_default_options(precision="mixed", separable_tensor_cores=tc))
        try:
            s.set_separable(dims, cdr_axes(dims, beta))
            x, iters, rel = s.shifted_solve(sigma, r)
        finally:
            s.close()
        assert rel <= 1e-12
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
        out.append(iters)
    assert abs(out[0] - out[1]) <= 1, out


@pytest.mark.gpu
def test_set_separable_rejects_bad_input(simlib):
    from workloads import cdr_axes, diag_csr

    A = cdr_csr((8, 8), (1.0, 0.5))
    s = simlib.Sim(A, None)
    with pytest.raises(simlib.SimError) as e:
        s.set_separable((8, 9), cdr_axes((8, 9), (1.0, 0.5)))  # product != n
    assert e.value.status == 1
    s.close()
    s = simlib.Sim(A, diag_csr(np.linspace(1.0, 2.0, 64)))
    with pytest.raises(simlib.SimError) as e:
        s.set_separable((8, 8), cdr_axes((8, 8), (1.0, 0.5)))  # B is not b·I
    assert e.value.status == 1
    s.close()


def _run_separable(simlib, w, precision):
    opt = simlib.sim_default_options(precision=precision, **w.options)
    s = simlib.Sim(w.A, None, opt)
    try:
        s.set_separable(*w.separable)
        s.set_region(w.region, w.f)
        s.solve_all_levels()
        eig = s.eigenvalues()
        mult = s.multiplicity()
        st = s.stats()
    finally:
        s.close()
    return eig, mult, st


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_simm_cdr2d_separable_matches_oracle(simlib, precision):
    w = config_cdr2d(30, 8)
    ref = S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))
    eig, mult, st = _run_separable(simlib, w, precision)
    assert eig.size == ref.eigenvalues.size == w.expected_count
    assert np.max(np.abs(eig - ref.eigenvalues)) <= 1e-6
    assert np.array_equal(mult, ref.multiplicities)
    assert st["num_shifts"] == len(ref.shifts)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_simm_cdr3d_separable_matches_oracle(simlib, cdr3d_small, precision):
    w, ref = cdr3d_small
    eig, mult, st = _run_separable(simlib, w, precision)
    assert eig.size == ref.eigenvalues.size
    assert np.max(np.abs(eig - ref.eigenvalues)) <= 1e-6
    assert np.array_equal(mult, ref.multiplicities)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_simm_cdr2d_full_size_matches_oracle_record(simlib, precision):
    """n = 250,000 (the 2-D convection–diffusion–reaction workload at full
    size): levels, shifts, eigenvalues and multiplicities equal to the
    oracle's run recorded by tests/golden/make_cdr2d_record.py."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "cdr2d500_record.json")) as fh:
        ref = json.load(fh)
    w = config_cdr2d()
    opt = simlib.sim_default_options(precision=precision, **w.options)
    s = simlib.Sim(w.A, None, opt)
    try:
        s.set_separable(*w.separable)
        s.set_region(w.region, w.f)
        marked = s.solve_all_levels()
        eig = s.eigenvalues()
        mult = s.multiplicity()
        st = s.stats()
    finally:
        s.close()
    assert [ref["level_counts"][0]] + [4 * m for m in marked[:-1]] == ref["level_counts"]
    assert st["num_shifts"] == ref["num_shifts"]
    est = np.array(ref["estimate_re"]) + 1j * np.array(ref["estimate_im"])
    assert eig.size == est.size == w.expected_count
    assert np.max(np.abs(eig - est)) <= 1e-9
    assert np.array_equal(mult, ref["multiplicity"])


@pytest.mark.gpu
def test_cdr3d_full_size_eigenpairs_have_small_residuals(simlib):
    """n = 10^6 (the 3-D workload at full size, 15-unit sub-region), where no
    oracle runs: every located eigenvalue, Ritz-refined (Sec. 3.2), with its
    projection P f (Remark 3.5) is an eigenpair of A to a small backward error
    ||A x - λ x|| / (|λ| ||x||), and each refined value lies within the
    precision h0 of its square's estimate."""
    w = config_cdr3d(100, 15.0)
    opt = simlib.sim_default_options(precision="mixed", **w.options)
    s = simlib.Sim(w.A, None, opt)
    try:
        s.set_separable(*w.separable)
        s.set_region(w.region, w.f)
        s.solve_all_levels()
        eig = s.eigenvalues()
        mult = s.multiplicity()
        ref, flag = s.refine()
        assert eig.size >= 100 and np.all(mult == 1) and flag.all()
        assert np.max(np.abs(ref - eig)) <= w.options["h0"]
        for c in np.random.default_rng(2).choice(eig.size, 6, replace=False):
            x = torch.from_numpy(s.projection(int(c))).cuda()
            r = s.apply_shifted(ref[c], x)
            xn = float(torch.linalg.norm(x))
            assert xn > 0.0
            assert float(torch.linalg.norm(r)) <= 1e-8 * abs(ref[c]) * xn, (c, ref[c])
    finally:
        s.close()
