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


def _p12_record():
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "batch_p12_record.json")) as fh:
        return json.load(fh)


def test_new_shifts_in_levels_record_matches_closed_form():
    """Pencil 12 of the 64-pencil workload: with new shifts at the levels the
    oracle locates exactly the closed-form eigenvalues of its region (the
    record of tests/golden/make_batch_p12_record.py)."""
    from workloads import cd2d_eigenvalues

    ref = _p12_record()
    w = config_batch(64).pencils[ref["pencil"]]
    N = w.separable[0][0]
    h = 1.0 / (N + 1)
    beta = tuple(float(((a[2] - a[0]) * h).real) for a in w.separable[1])
    lam = np.sort(cd2d_eigenvalues(N, beta).real)
    lo, hi = w.region[:2]
    inside = lam[(lam > lo) & (lam < hi)]
    est = np.sort(np.array(ref["estimate_re"]))
    assert est.size == inside.size == ref["expected_count"]
    assert np.max(np.abs(est - inside)) <= 1e-6
    assert np.max(np.abs(ref["estimate_im"])) <= 1e-6
    assert ref["num_shifts"] > ref["initial_shifts"] and ref["unresolvable_final"] == 0


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_new_shifts_in_levels_gpu_matches_oracle_record(simlib, precision):
    """The same pencil on the GPU, alone and in a batch with a smaller pencil:
    levels, shifts and every estimate equal to the oracle's record."""
    ref = _p12_record()
    b = config_batch(64)
    w = b.pencils[ref["pencil"]]
    opt = simlib.sim_default_options(precision=precision, new_shifts_in_levels=1, **w.options)
    s = simlib.Sim(w.A, None, opt)
    try:
        s.set_separable(*w.separable)
        s.set_region(w.region, w.f)
        marked = s.solve_all_levels()
        eig = s.eigenvalues()
        st = s.stats()
    finally:
        s.close()
    assert [ref["level_counts"][0]] + [4 * m for m in marked[:-1]] == ref["level_counts"]
    assert st["num_shifts"] == ref["num_shifts"]
    est = np.array(ref["estimate_re"]) + 1j * np.array(ref["estimate_im"])
    assert eig.size == est.size
    assert np.max(np.abs(eig - est)) <= 1e-9
    small = _small_batch().pencils[0]
    bt = simlib.Batch([small.A, w.A], None, opt)
    try:
        bt.set_separable(0, *small.separable)
        bt.set_separable(1, *w.separable)
        bt.set_regions([small.region, w.region], [small.f, w.f])
        bt.solve_all_levels()
        assert np.array_equal(bt.eigenvalues(1), eig)
        assert bt.stats(1)["num_shifts"] == ref["num_shifts"]
    finally:
        bt.close()
