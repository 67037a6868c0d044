"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
closed forms and exact inertia counts."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

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


def _csr_arrays(M):
    return (M.indptr, M.indices, M.data)


def _pencil_small():
    from workloads import cd2d_csr

    A = cd2d_csr(12, (1.0, 0.5))
    bd = np.random.default_rng(3).uniform(1.0, 2.0, A.n)
    return A, bd


# ---------------------------------------------------------------------------
def test_random_vectors_match_oracle_philox(simlib):
    from oracle.philox import random_vectors

    for seed, n, k, first in ((0x5EED, 1000, 3, 0), (7, 1537, 2, 5)):
        g = simlib.random_vectors(seed, n, k, first).cpu().numpy()
        ref = random_vectors(seed, n, k, first).T
        assert np.max(np.abs(g - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_apply_shifted_matches_scipy(simlib):
    from workloads import diag_csr

    A, bd = _pencil_small()
    B = diag_csr(bd)
    s = simlib.Sim(A, B)
    x = np.random.default_rng(1).standard_normal(A.n) + 1j * np.random.default_rng(2).standard_normal(A.n)
    sigma = 850.0 + 0.2j
    y = s.apply_shifted(sigma, torch.from_numpy(x).cuda()).cpu().numpy()
    ref = (A.to_scipy() - sigma * B.to_scipy()) @ x
    assert np.max(np.abs(y - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shifted_solve_matches_sparse_lu(simlib, precision):
    from workloads import block_diag_csr, jordan_csr, diag_csr

    A0, bd = _pencil_small()
    A = block_diag_csr(A0, jordan_csr([900.0 + 0.35j, 1300.0 + 0.35j], 4, 1e-7))  # ragged last block
    B = diag_csr(np.concatenate([bd, np.ones(8)]))
    s = simlib.Sim(A, B, simlib.sim_default_options(precision=precision))
    r = np.random.default_rng(4).standard_normal(A.n) + 0.5j
    sigma = 905.3 + 0.2j
    x, iters, rel = s.shifted_solve(sigma, torch.from_numpy(r).cuda())
    x = x.cpu().numpy()
    K = (A.to_scipy() - sigma * B.to_scipy()).tocsc()
    ref = spla.splu(K).solve(r)
    assert rel <= 1e-12
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert iters >= 1


def _cd2d_rect(nx, ny, beta=(1.0, 0.5)):
    """-Δu + β·∇u on an nx × ny interior grid of the unit square, x fastest:
    band half-width nx."""
    def d1(N, b):
        h = 1.0 / (N + 1)
        return sp.diags([(-1 / h**2 - b / (2 * h)) * np.ones(N - 1), 2 / h**2 * np.ones(N),
                         (-1 / h**2 + b / (2 * h)) * np.ones(N - 1)], [-1, 0, 1])
    A = sp.kron(sp.identity(ny), d1(nx, beta[0])) + sp.kron(d1(ny, beta[1]), sp.identity(nx))
    return sp.csr_matrix(A, dtype=np.complex128)


@pytest.mark.parametrize("precision,nx", [("fp64", 340), ("mixed", 470)])
def test_shifted_solve_single_cta_factorisation(simlib, precision, nx):
    """Blocks of side nx = 340 (complex128) or 470 (complex64) do not fit a
    cluster's shared memory: the single-CTA factorisation runs instead."""
    A = _cd2d_rect(nx, 3)
    A.sort_indices()
    s = simlib.Sim(_csr_arrays(A), None, simlib.sim_default_options(precision=precision))
    assert s.stats()["block_size"] == nx
    r = np.random.default_rng(11).standard_normal(A.shape[0]) + 0.25j
    sigma = 1.2e5 + 0.3j
    x, iters, rel = s.shifted_solve(sigma, torch.from_numpy(r).cuda())
    ref = spla.splu((A - sigma * sp.identity(A.shape[0])).tocsc()).solve(r)
    assert rel <= 1e-12
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
    s.close()


def _perturbed_spread(S, ks, centers, sides, name, trials=3, rel=4e-16):
    """How far rounding-size perturbations of H move the oracle's outputs:
    the conditioning bound a correct GPU result must stay within."""
    rng = np.random.default_rng(123)
    i0, r0 = S.evaluate_squares(ks, centers, sides, name)
    di, dr = np.zeros_like(i0), np.zeros_like(r0)
    for _ in range(trials):
        E = rng.standard_normal(ks.H.shape) + 1j * rng.standard_normal(ks.H.shape)
        kp = S.KrylovSpace(ks.sigma, ks.H * (1 + rel * E) * (ks.H != 0), ks.beta, ks.m_eff)
        i1, r1 = S.evaluate_squares(kp, centers, sides, name)
        di = np.maximum(di, np.abs(i1 - i0))
        dr = np.maximum(dr, np.abs(r1 - r0))
    return i0, r0, di, dr


def test_eval_squares_with_oracle_krylov_space(simlib):
    from oracle import simm as S
    from workloads import config_small

    w = config_small()
    ks = S.cayley_arnoldi(w.A.to_scipy(), sp.identity(w.A.n, format="csr", dtype=complex), 3990.0 + 0.2j, w.f, 50)
    rng = np.random.default_rng(9)
    centers = rng.uniform(3950, 4030, 300) + 1j * rng.uniform(-0.3, 0.7, 300)
    sides = 2.0 ** -rng.integers(0, 20, 300)
    for scale, name in ((0, "solution"), (1, "beta")):
        ind, rho = simlib.eval_squares(ks.H, ks.m_eff, ks.beta, ks.sigma, centers, sides, scale)
        ind_o, rho_o, di, dr = _perturbed_spread(S, ks, centers, sides, name)
        ok = np.isfinite(ind_o)
        # within 100x the spread that rounding-size perturbations of H produce (plus 1e-11)
        assert np.all(np.abs(ind[ok] - ind_o[ok]) <= 100 * di[ok] + 1e-11 * np.maximum(1.0, ind_o[ok]))
        okr = np.isfinite(rho_o)
        assert np.all(np.abs(rho[okr] - rho_o[okr]) <= 100 * dr[okr] + 1e-9 * rho_o[okr] + 1e-300)
        # and the decisions of Defs. 3.1-3.2 agree away from near-ties
        clear = (np.abs(np.log10(np.maximum(rho_o, 1e-300)) + 8.0) > 0.01) & (100 * dr < 0.5 * np.abs(rho_o - 1e-8))
        assert np.array_equal((rho <= 1e-8)[clear], (rho_o <= 1e-8)[clear])
        cl = ok & (np.abs(ind_o - 0.05) > 100 * di + 1e-9)
        assert np.array_equal((ind > 0.05)[cl], (ind_o > 0.05)[cl])
    # squares the space resolves (Def. 3.1) and that are not tiny: tight agreement
    ind, rho = simlib.eval_squares(ks.H, ks.m_eff, ks.beta, ks.sigma, centers, sides, 0)
    ind_o, rho_o = S.evaluate_squares(ks, centers, sides, "solution")
    sel = (rho_o <= 1e-8) & (sides >= 1e-3) & (ind_o > 1e-2)
    assert sel.sum() >= 5
    assert np.all(np.abs(ind[sel] - ind_o[sel]) <= 1e-7 * ind_o[sel])


def test_krylov_space_matches_oracle(simlib):
    from oracle import simm as S
    from workloads import config_small

    w = config_small()
    s = simlib.Sim(w.A, None)
    s.set_region(w.region, w.f)
    sigma, H, beta, meff = s.get_shift(0)
    ks = S.cayley_arnoldi(w.A.to_scipy(), sp.identity(w.A.n, format="csr", dtype=complex), sigma, w.f, 50)
    assert meff == ks.m_eff == 50
    assert abs(beta - ks.beta) <= 1e-11 * ks.beta
    # leading columns agree to rounding; the subdiagonal is real and positive
    assert np.max(np.abs(H[:12, :10] - ks.H[:12, :10])) <= 1e-8 * np.max(np.abs(ks.H))
    assert np.all(np.diag(H, -1).real > 0)
    # indicators of squares near σ computed from either space agree
    centers = sigma + np.linspace(-15, 15, 61) + 0.05j
    i_gpu, _ = S.evaluate_squares(S.KrylovSpace(sigma, H, beta, meff), centers, np.full(61, 0.5))
    i_ora, _ = S.evaluate_squares(ks, centers, np.full(61, 0.5))
    assert np.all(np.abs(i_gpu - i_ora) <= 1e-6 * np.maximum(1.0, i_ora))


@pytest.fixture(scope="module")
def small_oracle():
    from oracle import simm as S
    from workloads import config_small

    w = config_small()
    return w, S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_simm_small_convection_diffusion(simlib, small_oracle, precision):
    w, ref = small_oracle
    opt = simlib.sim_default_options(precision=precision, **w.options)
    eig, mult, st = simlib.run(w.A, None, w.region, w.f, opt)
    assert eig.size == ref.eigenvalues.size == w.expected_count == 50
    assert np.max(np.abs(eig - ref.eigenvalues)) <= 1e-6
    assert np.max(np.abs(np.sort(eig.real) - np.sort(w.reference_eigs.real))) <= 1e-6
    assert np.array_equal(mult, ref.multiplicities)
    assert st["unresolvable_final"] == 0
    assert st["max_inner_residual"] <= 100 * opt.mult_inner_tol  # worst accepted inner solve
    assert st["loose_inner_solves"] == 0


def test_simm_jordan_multiplicity(simlib):
    from oracle import simm as S
    from workloads import config_jordan_small

    w = config_jordan_small()
    ref = S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options))
    eig, mult, _ = simlib.run(w.A, None, w.region, w.f, simlib.sim_default_options(**w.options))
    assert eig.size == ref.eigenvalues.size == w.reference_eigs.size
    assert np.max(np.abs(eig - ref.eigenvalues)) <= 1e-6
    assert np.array_equal(mult, ref.multiplicities)
    assert np.array_equal(mult, w.reference_mult)


@pytest.mark.parametrize("case", ["small", "jordan", "generalized"])
def test_schur_level_solver_equals_direct_solves(simlib, case):
    """level_solver 1 (Schur form of H_m per shift, one triangular solve per
    node, Sec. 3.2) and level_solver 0 (Gaussian elimination of I + (σ - z)H_m
    at every node) evaluate the same quantities: the same squares are marked at
    every level, the located eigenvalues are the same square centres and the
    shift retries are the same (the Schur path evaluates a square its own shift
    leaves against every shift and picks the one the direct order would)."""
    import scipy.linalg as sla

    from workloads import cd2d_csr, config_jordan_small, config_small, diag_csr

    if case == "generalized":
        A = cd2d_csr(15, (1.0, 0.5))
        bd = np.random.default_rng(11).uniform(1.0, 2.0, A.n)
        lr = np.sort(sla.eigvals(A.to_dense(), np.diag(bd)).real)
        B, region, options = diag_csr(bd), (0.5 * (lr[99] + lr[100]), 0.5 * (lr[119] + lr[120]), -0.3, 0.7), {}
        f = np.random.default_rng(12).standard_normal(A.n) + 0j
    else:
        w = config_small() if case == "small" else config_jordan_small()
        A, B, region, f, options = w.A, w.B, w.region, w.f, w.options
    out = []
    for solver in (0, 1):
        opt = simlib.sim_default_options(level_solver=solver, **options)
        s = simlib.Sim(A, B, opt)
        try:
            s.set_region(region, f)
            marked = s.solve_all_levels()
            out.append((marked, s.eigenvalues(), s.multiplicity(), s.stats()))
        finally:
            s.close()
    (m0, e0, u0, st0), (m1, e1, u1, st1) = out
    assert m0 == m1
    assert np.array_equal(e0, e1)
    assert np.array_equal(u0, u1)
    assert st0["shift_retries"] == st1["shift_retries"]
    assert st0["direct_level_evaluations"] == st0["squares_evaluated"]
    assert st1["direct_level_evaluations"] < st1["squares_evaluated"] // 2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multiplicity_single_pass_equals_cgs2(simlib, precision):
    # The multiplicity spaces use one classical Gram-Schmidt pass by default (the
    # algorithm as printed in Sec. 2); reorthogonalising them (mult_reorth = 1, CGS2
    # as in the location spaces) gives the same eigenvalues and multiplicities.
    from workloads import config_jordan_small

    w = config_jordan_small()
    runs = [simlib.run(w.A, None, w.region, w.f,
                       simlib.sim_default_options(precision=precision, mult_reorth=r, **w.options))
            for r in (0, 1)]
    (eig0, mult0, st0), (eig1, mult1, st1) = runs
    assert np.array_equal(eig0, eig1)  # location does not depend on the option
    assert np.array_equal(mult0, mult1)
    assert np.array_equal(mult0, w.reference_mult)


def test_large_n_uses_multi_kernel_gram_schmidt(simlib):
    # n = 41,209 is beyond the single-launch Gram-Schmidt's range (n <= 40,960),
    # so the four-kernel version with partial sums in global memory runs here;
    # the eigenvalues are checked against the closed form.
    from workloads import cd2d_csr, cd2d_eigenvalues, complex_gaussian
    from workloads.configs import max_gap_window, window_region

    N = 203
    A = cd2d_csr(N, (1.0, 0.5))
    lr = np.sort(cd2d_eigenvalues(N, (1.0, 0.5)).real)
    start = max_gap_window(lr, 6, lr.size // 2 - 2000, lr.size // 2 + 2000)
    region = window_region(lr, start, 6)
    inside = lr[(lr > region[0]) & (lr < region[1])]
    eig, mult, _ = simlib.run(A, None, region, complex_gaussian(A.n, 3),
                              simlib.sim_default_options(precision="mixed", h0=1e-6))
    assert eig.size == inside.size == 6
    assert np.max(np.abs(np.sort(eig.real) - inside)) <= 1e-6
    assert np.all(mult == 1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ritz_refinement_matches_oracle_and_closed_form(simlib, precision):
    # Sec. 3.2: refined eigenvalues σ + 1/d from the Hessenberg QR on the GPU,
    # against the oracle's refinement (numpy eigvals) and the closed form.
    from oracle import simm as S
    from workloads import config_small

    w = config_small()
    sim = S.SimM(w.A.to_scipy(), None, S.Options(**w.options))
    sim.set_region(w.region, w.f)
    sim.solve_levels()
    sim.merge()
    ref_o, flag_o = sim.refine()
    s = simlib.Sim(w.A, None, simlib.sim_default_options(precision=precision, **w.options))
    try:
        s.set_region(w.region, w.f)
        s.solve_all_levels()
        eig = s.eigenvalues()
        ref_g, flag_g = s.refine()
        ref_g2, _ = s.refine()  # repeatable
    finally:
        s.close()
    truth = np.sort_complex(w.reference_eigs)
    assert eig.size == ref_g.size == ref_o.size == truth.size
    assert np.array_equal(flag_g, flag_o) and flag_g.all()
    assert np.array_equal(ref_g, ref_g2)
    assert np.max(np.abs(ref_g - ref_o)) <= 2e-8
    assert np.max(np.min(np.abs(ref_g[:, None] - truth[None, :]), axis=1)) <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_projection_vector_matches_oracle(simlib, precision):
    # P f of a located eigenvalue (an eigenvector for a simple one), GPU against
    # the oracle's, and its eigen-residual with the refined eigenvalue.
    from oracle import simm as S
    from workloads import config_small

    w = config_small()
    A = w.A.to_scipy()
    sim = S.SimM(A, None, S.Options(**w.options))
    sim.set_region(w.region, w.f)
    sim.solve_levels()
    sim.merge()
    s = simlib.Sim(w.A, None, simlib.sim_default_options(precision=precision, **w.options))
    try:
        s.set_region(w.region, w.f)
        s.solve_all_levels()
        s.eigenvalues()
        ref, _ = s.refine()
        for c in (0, 17, 49):
            x = s.projection(c)
            xo = sim.projection(c)
            assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
            assert np.linalg.norm(A @ x - ref[c] * x) <= 1e-10 * abs(ref[c]) * np.linalg.norm(x)
        with pytest.raises(simlib.SimError):
            s.projection(10**6)
    finally:
        s.close()


def test_simm_generalized_pencil_vs_dense_qz(simlib):
    import scipy.linalg as sla

    from workloads import cd2d_csr, diag_csr

    N = 15
    A0 = cd2d_csr(N, (1.0, 0.5))
    bd = np.random.default_rng(11).uniform(1.0, 2.0, A0.n)
    lam = sla.eigvals(A0.to_dense(), np.diag(bd))
    lr = np.sort(lam.real)
    lo, hi = 0.5 * (lr[99] + lr[100]), 0.5 * (lr[119] + lr[120])
    f = np.random.default_rng(12).standard_normal(A0.n) + 0j
    eig, mult, _ = simlib.run(A0, diag_csr(bd), (lo, hi, -0.3, 0.7), f)
    assert eig.size == 20
    assert np.max(np.abs(np.sort(eig.real) - np.sort(lam[(lam.real > lo) & (lam.real < hi)].real))) <= 1e-6
    assert np.all(mult == 1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_refinement_and_projection_on_generalized_pencil(simlib, precision):
    # B ≠ I: GPU refined eigenvalues against dense QZ and the oracle, and P f
    # against A x = λ B x and the oracle's P f.
    import scipy.linalg as sla

    from oracle import simm as S
    from workloads import cd2d_csr, diag_csr

    N = 15
    A0 = cd2d_csr(N, (1.0, 0.5))
    bd = np.random.default_rng(11).uniform(1.0, 2.0, A0.n)
    Ad, Bd = A0.to_dense(), np.diag(bd)
    lam = sla.eigvals(Ad, Bd)
    lr = np.sort(lam.real)
    lo, hi = 0.5 * (lr[99] + lr[100]), 0.5 * (lr[119] + lr[120])
    inside = lam[(lam.real > lo) & (lam.real < hi)]
    region = (lo, hi, -0.3, 0.7)
    f = np.random.default_rng(12).standard_normal(A0.n) + 0j
    sim = S.SimM(A0.to_scipy(), diag_csr(bd).to_scipy(), S.Options(h0=1e-6))
    sim.set_region(region, f)
    sim.solve_levels()
    sim.merge()
    ref_o, flag_o = sim.refine()
    s = simlib.Sim(A0, diag_csr(bd), simlib.sim_default_options(precision=precision, h0=1e-6))
    try:
        s.set_region(region, f)
        s.solve_all_levels()
        s.eigenvalues()
        ref, flag = s.refine()
        assert flag.all() and np.array_equal(flag, flag_o)
        assert np.max(np.min(np.abs(ref[:, None] - inside[None, :]), axis=1)) <= 1e-8
        assert np.max(np.abs(ref - ref_o)) <= 2e-8
        for c in (0, 9, 19):
            x = s.projection(c)
            assert np.linalg.norm(x - sim.projection(c)) <= 1e-8 * np.linalg.norm(x)
            assert np.linalg.norm(Ad @ x - ref[c] * (Bd @ x)) <= 1e-8 * abs(ref[c]) * np.linalg.norm(Bd @ x)
    finally:
        s.close()


def test_simm_laplacian_degenerate_multiplicity(simlib):
    from oracle import simm as S
    from workloads import cd2d_csr

    N = 8
    A = cd2d_csr(N, (0.0, 0.0))
    ev = np.sort(np.linalg.eigvalsh(A.to_dense().real))
    h = 1.0 / (N + 1)
    c = 4.0 / h**2
    uniq = np.unique(np.round(ev, 6))
    j = int(np.argmin(np.abs(uniq - c)))
    lo, hi = 0.5 * (uniq[j - 3] + uniq[j - 2]), 0.5 * (uniq[j + 2] + uniq[j + 3])
    f = np.random.default_rng(13).standard_normal(A.n) + 0j
    ref = S.sim_m(A.to_scipy(), None, (lo, hi, -0.4, 0.6), f, S.Options())
    eig, mult, _ = simlib.run(A, None, (lo, hi, -0.4, 0.6), f)
    assert np.max(np.abs(eig - ref.eigenvalues)) <= 1e-6
    assert np.array_equal(mult, ref.multiplicities)
    assert mult.max() == N  # the eigenvalue 4/h^2 has multiplicity N


def test_empty_region_and_state_errors(simlib):
    from workloads import cd2d_csr, complex_gaussian

    A = cd2d_csr(10, (1.0, 0.5))
    s = simlib.Sim(A, None)
    with pytest.raises(simlib.SimError) as e:
        s.solve_level()
    assert e.value.status == 2  # SIM_ERR_BAD_STATE
    s.set_region((-50.0, -10.0, -1.0, 1.0), complex_gaussian(A.n, 0))  # left of the spectrum
    s.solve_all_levels()
    assert s.eigenvalues().size == 0
    assert s.multiplicity().size == 0
    with pytest.raises(simlib.SimError) as e:
        s.solve_level()
    assert e.value.status == 2


def test_invalid_csr_is_rejected(simlib):
    bad = (np.array([0, 2, 3], np.int32), np.array([1, 0, 1], np.int32), np.ones(3, complex))  # unsorted row 0
    with pytest.raises(simlib.SimError) as e:
        simlib.Sim(bad, None)
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# the benchmark configuration at full size: n = 40,064, B diagonal, Jordan blocks
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module", params=["mixed", "fp64"])
def pencil_run(simlib, request):
    from workloads import config_pencil

    w = config_pencil()
    opt = simlib.sim_default_options(precision=request.param, **w.options)
    s = simlib.Sim(w.A, w.B, opt)
    try:
        s.set_region(w.region, w.f)
        marked = s.solve_all_levels()
        eig = s.eigenvalues()
        mult = s.multiplicity()
        st = s.stats()
    finally:
        s.close()
    st["marked_per_level"] = marked
    return w, eig, mult, st


def test_pencil_counts_and_multiplicities(pencil_run):
    from workloads.configs import jordan_eigs

    w, eig, mult, st = pencil_run
    assert int(mult.sum()) == w.expected_count == 564
    je = jordan_eigs(w.region)
    jd = np.abs(eig[:, None] - je[None, :])
    is_j = jd.min(axis=1) < 1e-3
    assert is_j.sum() == 16
    assert np.all(mult[is_j] == 4)
    assert np.all(mult[~is_j] == 1)
    assert np.max(jd.min(axis=0)) <= 1e-6
    assert np.max(np.abs(eig[~is_j].imag)) <= 1e-6  # the convection-diffusion pencil is real


def test_pencil_sampled_eigenvalues_by_inertia(pencil_run):
    from oracle.inertia import count_below
    from workloads.configs import pencil_parts

    w, eig, mult, st = pencil_run
    _, bd = pencil_parts(200, 1)
    real = np.sort(eig[np.abs(eig.imag) < 1e-3].real)
    rng = np.random.default_rng(0)
    for x in rng.choice(real, 6, replace=False):
        # exactly one eigenvalue of the pencil within 2e-6 of each sampled estimate
        assert count_below(200, (1.0, 0.5), bd, x + 2e-6) - count_below(200, (1.0, 0.5), bd, x - 2e-6) == 1



def test_pencil_levels_and_clusters_equal_the_oracle_record(pencil_run):
    """The oracle's location phase on the full pencil, recorded by
    tests/golden/make_pencil_levels.py: the same squares per level, shifts,
    unresolvable final squares and clusters, with every estimate equal."""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "pencil40064_levels.json")) as fh:
        ref = json.load(fh)
    w, eig, mult, st = pencil_run
    marked = st["marked_per_level"]
    evaluated = [ref["level_counts"][0]] + [4 * m for m in marked[:-1]]
    assert evaluated == ref["level_counts"]
    assert st["num_shifts"] == ref["num_shifts"]
    assert st["final_squares"] == ref["final_squares"] == marked[-1]
    assert st["unresolvable_final"] == ref["unresolvable_final"]
    est = np.array(ref["estimate_re"]) + 1j * np.array(ref["estimate_im"])
    assert eig.size == est.size == ref["clusters"]
    assert np.max(np.abs(eig - est)) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_screen_matches_oracle_on_the_same_krylov_space(simlib, precision):
    """Sec. 3.2 on the GPU (eigendecomposition of H_m, O(m) per point) against
    the oracle's formula and its direct Hessenberg solve, both fed the GPU's
    Krylov space of a normal matrix (well-conditioned eigenvectors)."""
    from oracle import simm as S
    from workloads import diag_csr

    rng = np.random.default_rng(12)
    lam = rng.uniform(0, 10, 80) + 1j * rng.uniform(-1, 1, 80)
    f = rng.standard_normal(80) + 1j * rng.standard_normal(80)
    s = simlib.Sim(diag_csr(lam), None, simlib.sim_default_options(precision=precision, h0=1e-3))
    s.set_region((3.0, 7.0, -0.7, 1.3), f)
    sigma, H, beta, meff = s.get_shift(0)
    ks = S.KrylovSpace(sigma, H[: meff + 1, :meff], beta, meff)
    near = lam[np.argsort(np.abs(lam - sigma))[:24]]
    z = np.concatenate([sigma + rng.uniform(-2, 2, 40) + 1j * rng.uniform(-1, 1, 40),
                        near + 0.02 * np.exp(2j * np.pi * rng.uniform(size=24))])
    ym, rho = s.residual_screen(0, z)
    ym_o, rho_o = S.screened_last_entry(ks, z)
    y, rho_d = S.projected_solve(ks, z, "beta")
    d, P, c1, rm = S.eig_decomposition(ks)
    scale = beta * np.sum(np.abs(rm * c1 / (1.0 + (sigma - z)[:, None] * d)), axis=-1)
    assert np.all(np.abs(ym - ym_o) <= 1e-9 * np.abs(ym_o) + 1e-11 * scale)
    assert np.all(np.abs(ym - y[:, -1]) <= 1e-9 * np.abs(y[:, -1]) + 1e-11 * scale)
    big = np.abs(ym_o) > 1e-6 * scale
    assert big.sum() >= 10
    assert np.max(np.abs(rho[big] - rho_d[big]) / rho_d[big]) <= 1e-8
    s.close()
