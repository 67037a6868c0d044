"""Batches of pencils (sim_batch_*): every pencil's squares of a level in one
evaluation launch.  Each pencil's result must equal the oracle's run on that
pencil alone, and the closed-form count of its region."""
import numpy as np
import pytest

from oracle import simm as S
from workloads.configs import config_batch


def _small_batch():
    return config_batch(6, n_lo=12, n_span=18, eig_lo=5, eig_hi=20)


@pytest.fixture(scope="module")
def batch_oracle():
    b = _small_batch()
    refs = [S.sim_m(w.A.to_scipy(), None, w.region, w.f, S.Options(**w.options)) for w in b.pencils]
    return b, refs


def test_oracle_batch_pencils_match_closed_form(batch_oracle):
    from workloads import cd2d_eigenvalues

    b, refs = batch_oracle
    for w, r in zip(b.pencils, refs):
        # the closed-form eigenvalues inside the region, each within h0
        N = w.separable[0][0]
        lam = np.sort(np.linalg.eigvals(w.A.to_scipy().toarray()).real)
        lo, hi = w.region[:2]
        inside = lam[(lam > lo) & (lam < hi)]
        assert r.eigenvalues.size == inside.size == w.expected_count
        assert np.max(np.abs(np.sort(r.eigenvalues.real) - inside)) <= 1e-6
        assert np.array_equal(r.multiplicities, np.ones(w.expected_count, dtype=np.int64))
        assert N * N == w.A.n


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def simlib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g

    g.build()
    import paper_2006_16117_gb300 as sim

    return sim


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_equals_oracle_per_pencil(simlib, batch_oracle, precision):
    b, refs = batch_oracle
    opt = simlib.sim_default_options(precision=precision, **b.pencils[0].options)
    bt = simlib.Batch([w.A for w in b.pencils], None, opt)
    try:
        for p, w in enumerate(b.pencils):
            bt.set_separable(p, *w.separable)
        bt.set_regions([w.region for w in b.pencils], [w.f for w in b.pencils])
        bt.solve_all_levels()
        for p, (w, r) in enumerate(zip(b.pencils, refs)):
            eig = bt.eigenvalues(p)
            mult = bt.multiplicity(p)
            assert eig.size == r.eigenvalues.size == w.expected_count
            assert np.max(np.abs(eig - r.eigenvalues)) <= 1e-6
            assert np.array_equal(mult, r.multiplicities)
    finally:
        bt.close()


@pytest.mark.gpu
def test_batch_equals_single_pencil_runs(simlib):
    """The batched level evaluation gives bit-identical eigenvalues to one
    handle per pencil (the same kernels on the same squares)."""
    b = _small_batch()
    opt = simlib.sim_default_options(precision="mixed", **b.pencils[0].options)
    bt = simlib.Batch([w.A for w in b.pencils], None, opt)
    try:
        for p, w in enumerate(b.pencils):
            bt.set_separable(p, *w.separable)
        bt.set_regions([w.region for w in b.pencils], [w.f for w in b.pencils])
        bt.solve_all_levels()
        for p, w in enumerate(b.pencils):
            s = simlib.Sim(w.A, None, opt)
            s.set_separable(*w.separable)
            s.set_region(w.region, w.f)
            s.solve_all_levels()
            assert np.array_equal(s.eigenvalues(), bt.eigenvalues(p))
            s.close()
    finally:
        bt.close()
