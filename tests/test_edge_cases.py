"""Edge cases of the method, on the oracle (pinned to closed forms or to an
invariant of its own unmerged output) and on the GPU (equal to the oracle):

* clusters closer than merge_radius are joined (Sec. 3.5 step 6, reading 15);
* a defective eigenvalue with a large Jordan coupling: the coarse rule's
  aliasing of the higher-order pole drives the indicator of Eq. DeltaSm below
  δ0, so the eigenvalue is not located — a property of the method that both
  sides must share;
* an eigenvalue exactly on a quadrature node (a corner shared by four
  squares, reading 2);
* an indicator within 1e-10 of δ0 (reading 18) on either side, including a
  level where no square is marked (an empty next level);
* an initial tiling that overhangs R (reading 8): eigenvalues in the overhang
  are located but not reported.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so

from oracle import simm as S
from workloads import block_diag_csr, complex_gaussian, diag_csr, jordan_csr

SQ = 1.0 / math.sqrt(2.0)


def _oracle(A, region, f, **kw):
    return S.sim_m(A.to_scipy(), None, region, f, S.Options(**kw))


# ---------------------------------------------------------------------------
# merge radius
# ---------------------------------------------------------------------------
MERGE_EIGS = np.array([0.4 + 0.3j, 0.4 + 0.3j + 2e-5, 0.8 + 0.7j, 5.0 + 5.0j])


def test_merge_radius_joins_close_clusters_oracle():
    A = diag_csr(MERGE_EIGS)
    f = complex_gaussian(A.n, 0)
    sep = _oracle(A, (0, 1, 0, 1), f, h0=1e-6)
    # two eigenvalues 2e-5 apart: separate 8-connected components at h0 = 1e-6
    assert sep.eigenvalues.size == 3
    assert np.max(np.abs(sep.eigenvalues - MERGE_EIGS[:3])) <= 1e-6
    assert np.array_equal(sep.multiplicities, [1, 1, 1])
    joined = _oracle(A, (0, 1, 0, 1), f, h0=1e-6, merge_radius=5e-5)
    assert joined.eigenvalues.size == 2
    # the joined estimate is the mean of all member centres: the size-weighted
    # mean of the two unmerged components' estimates
    n1, n2 = sep.cluster_size[:2]
    want = (n1 * sep.eigenvalues[0] + n2 * sep.eigenvalues[1]) / (n1 + n2)
    assert abs(joined.eigenvalues[0] - want) <= 1e-15 * abs(want)
    assert joined.cluster_size[0] == n1 + n2
    # both eigenvalues lie inside its multiplicity circle: multiplicity 2
    assert np.array_equal(joined.multiplicities, [2, 1])
    assert abs(joined.eigenvalues[1] - sep.eigenvalues[2]) == 0.0
    # a radius below the distance joins nothing
    small = _oracle(A, (0, 1, 0, 1), f, h0=1e-6, merge_radius=1e-5)
    assert np.array_equal(small.eigenvalues, sep.eigenvalues)


# ---------------------------------------------------------------------------
# defective eigenvalue, Jordan coupling nu
# ---------------------------------------------------------------------------
JORDAN_LAM = 0.45 + 0.55j
JORDAN_DIAG = np.array([0.2 + 0.2j, 0.7 + 0.6j, 3.0 + 3.0j])


def _jordan_pencil(nu):
    return block_diag_csr(diag_csr(JORDAN_DIAG), jordan_csr(np.array([JORDAN_LAM]), 4, nu))


def _jordan_indicator_closed_form(nu, f, c, s):
    """Ĩ from the explicit resolvent: diagonal part f_k/(d_k - z); Jordan part
    (λI + νN - z)^{-1} = Σ_{p=0}^{3} (-ν)^p N^p / (λ - z)^{p+1}."""
    r = s * SQ
    ang = np.arange(8) * (np.pi / 4)
    off = r * (np.cos(ang) + 1j * np.sin(ang))
    X = []
    for o in off:
        z = c + o
        x = np.zeros(7, dtype=complex)
        x[:3] = f[:3] / (JORDAN_DIAG - z)
        fj = f[3:]
        for i in range(4):  # row i of the Jordan block's resolvent applied to fj
            x[3 + i] = sum((-nu) ** p * fj[i + p] / (JORDAN_LAM - z) ** (p + 1) for p in range(4 - i))
        X.append(x)
    X = np.array(X)
    Y8 = (off / 8) @ X
    Y4 = (off[0::2] / 4) @ X[0::2]
    return np.linalg.norm(Y8) / np.linalg.norm(Y4)


@pytest.mark.parametrize("nu", [1e-7, 1.0])
def test_defective_indicator_matches_explicit_jordan_resolvent(nu):
    A = _jordan_pencil(nu)
    f = complex_gaussian(A.n, 0)
    sigma = 0.5 + 0.5j
    ks = S.cayley_arnoldi(A.to_scipy(), _eye(A.n), sigma, f, 50)
    assert ks.m_eff == 7  # exact Krylov space: n = 7 <= m
    for s in (1.0, 0.5, 0.25, 0.125, 1 / 64):
        c = JORDAN_LAM + 0.1 * s * (1 + 1j)
        got, _ = S.evaluate_squares(ks, np.array([c]), np.array([s]))
        want = _jordan_indicator_closed_form(nu, f, c, s)
        assert abs(got[0] - want) <= 1e-9 * want, (s, got[0], want)
    # the coarse rule aliases the fourth-order pole: with nu = 1 the indicator of
    # a small square around the eigenvalue falls below δ0 = 0.05; with a tiny nu
    # it stays near 1 (Ĩ = 1/|1 + u^4| for a simple pole)
    small = _jordan_indicator_closed_form(nu, f, JORDAN_LAM + 0.01 * (1 + 1j), 0.25)
    assert (small < 0.05) if nu == 1.0 else (small > 0.9)


def _eye(n):
    import scipy.sparse as sp

    return sp.identity(n, dtype=complex, format="csr")


def test_strongly_defective_eigenvalue_is_not_located_oracle():
    f = complex_gaussian(7, 0)
    weak = _oracle(_jordan_pencil(1e-7), (0, 1, 0, 1), f, h0=1e-4, merge_radius=1e-3)
    assert weak.eigenvalues.size == 3
    assert np.max(np.abs(weak.eigenvalues - np.array([0.2 + 0.2j, JORDAN_LAM, 0.7 + 0.6j]))) <= 1e-4
    assert np.array_equal(weak.multiplicities, [1, 4, 1])
    strong = _oracle(_jordan_pencil(1.0), (0, 1, 0, 1), f, h0=1e-4, merge_radius=1e-3)
    assert strong.eigenvalues.size == 2
    assert np.max(np.abs(strong.eigenvalues - np.array([0.2 + 0.2j, 0.7 + 0.6j]))) <= 1e-4
    assert np.array_equal(strong.multiplicities, [1, 1])


# ---------------------------------------------------------------------------
# eigenvalue on a node; overhanging tiling
# ---------------------------------------------------------------------------
NODE_EIGS = np.array([1.0 + 1.0j, 3.3 + 2.6j, 10.0 + 10.0j])   # 1+1i: a corner from level 3 on
NODE_REGION = (0.0, 4.0, 0.0, 4.0)
OVER_EIGS = np.array([0.5 + 0.5j, 1.7 + 0.3j, 2.7 + 0.5j, 9.0 + 9.0j])
OVER_REGION = (0.0, 2.5, 0.0, 1.0)   # init_side 1: three columns, the last covers [2, 3]


def test_eigenvalue_on_a_node_oracle():
    A = diag_csr(NODE_EIGS)
    r = _oracle(A, NODE_REGION, complex_gaussian(A.n, 0), h0=1e-6)
    assert r.eigenvalues.size == 2
    # the four squares sharing the corner are marked symmetrically: the
    # estimate is the node itself
    assert abs(r.eigenvalues[0] - NODE_EIGS[0]) <= 1e-12
    assert abs(r.eigenvalues[1] - NODE_EIGS[1]) <= 1e-6
    assert np.array_equal(r.multiplicities, [1, 1])


def test_overhanging_tiling_filters_to_region_oracle():
    A = diag_csr(OVER_EIGS)
    r = _oracle(A, OVER_REGION, complex_gaussian(A.n, 0), h0=1e-6, init_side=1.0)
    assert r.level_counts[0] == 3
    assert r.eigenvalues.size == 2  # 2.7+0.5i lies in the overhang, outside R
    assert np.max(np.abs(r.eigenvalues - OVER_EIGS[:2])) <= 1e-6
    assert np.array_equal(r.multiplicities, [1, 1])


# ---------------------------------------------------------------------------
# indicator within 1e-10 of δ0
# ---------------------------------------------------------------------------
def _near_threshold_pencil(delta):
    """Two eigenvalues outside R = [0,1]²: one placed on the real line through
    the centre so that the single level-1 square has Ĩ = δ0 + delta (closed
    form of the diagonal case), one far away."""
    c, r = 0.5 + 0.5j, SQ
    f = complex_gaussian(2, 0)
    far = 40.0 + 40.0j

    def ind(u):
        lam = np.array([c + u * r, far])
        uu = (lam - c) / r
        return np.linalg.norm(f / (1 - uu**8)) / np.linalg.norm(f / (1 - uu**4))

    u = so.brentq(lambda u: ind(u) - (0.05 + delta), 1.5, 3.0, xtol=1e-15, rtol=1e-15)
    return np.array([c + u * r, far]), f, ind(u)


@pytest.mark.parametrize("delta", [1e-10, -1e-10])
def test_near_threshold_indicator_oracle(delta):
    lam, f, want = _near_threshold_pencil(delta)
    assert abs(want - (0.05 + delta)) <= 1e-13
    A = diag_csr(lam)
    ks = S.cayley_arnoldi(A.to_scipy(), _eye(2), 0.5 + 0.5j, f, 50)
    got, _ = S.evaluate_squares(ks, np.array([0.5 + 0.5j]), np.array([1.0]))
    assert abs(got[0] - want) <= 1e-13
    r = _oracle(A, (0, 1, 0, 1), f, h0=1e-3)
    assert r.level_counts[:2] == ([1, 4] if delta > 0 else [1, 0])
    assert r.eigenvalues.size == 0


# ---------------------------------------------------------------------------
# the same cases on the GPU, equal to the oracle
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


def _gpu_vs_oracle(simlib, A, region, precision="fp64", **kw):
    f = complex_gaussian(A.n, 0)
    ref = _oracle(A, region, f, **kw)
    opt = simlib.sim_default_options(precision=precision, **kw)
    s = simlib.Sim(A, None, opt)
    try:
        s.set_region(region, f)
        marked = s.solve_all_levels()
        eig = s.eigenvalues()
        mult = s.multiplicity()
    finally:
        s.close()
    # squares evaluated per level: 4 children per marked square
    evaluated = [ref.level_counts[0]] + [4 * m for m in marked[:-1]]
    assert evaluated == list(ref.level_counts)
    assert eig.size == ref.eigenvalues.size
    if eig.size:
        assert np.max(np.abs(eig - ref.eigenvalues)) <= 1e-12 * max(1.0, np.max(np.abs(eig)))
    assert np.array_equal(mult, ref.multiplicities)
    return eig, mult


@pytest.mark.gpu
@pytest.mark.parametrize("radius", [0.0, 1e-5, 5e-5])
def test_merge_radius_gpu(simlib, radius):
    eig, mult = _gpu_vs_oracle(simlib, diag_csr(MERGE_EIGS), (0, 1, 0, 1), h0=1e-6, merge_radius=radius)
    assert eig.size == (2 if radius > 2e-5 else 3)


@pytest.mark.gpu
@pytest.mark.parametrize("nu", [1e-7, 1.0])
def test_defective_eigenvalue_gpu(simlib, nu):
    eig, mult = _gpu_vs_oracle(simlib, _jordan_pencil(nu), (0, 1, 0, 1), h0=1e-4, merge_radius=1e-3)
    assert eig.size == (3 if nu < 1 else 2)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_eigenvalue_on_a_node_gpu(simlib, precision):
    eig, _ = _gpu_vs_oracle(simlib, diag_csr(NODE_EIGS), NODE_REGION, precision, h0=1e-6)
    assert abs(eig[0] - NODE_EIGS[0]) <= 1e-12


@pytest.mark.gpu
def test_overhanging_tiling_gpu(simlib):
    eig, _ = _gpu_vs_oracle(simlib, diag_csr(OVER_EIGS), OVER_REGION, h0=1e-6, init_side=1.0)
    assert eig.size == 2


@pytest.mark.gpu
@pytest.mark.parametrize("delta", [1e-10, -1e-10])
def test_near_threshold_indicator_gpu(simlib, delta):
    lam, f, want = _near_threshold_pencil(delta)
    A = diag_csr(lam)
    ks = S.cayley_arnoldi(A.to_scipy(), _eye(2), 0.5 + 0.5j, f, 50)
    ind, _ = simlib.eval_squares(ks.H, ks.m_eff, ks.beta, ks.sigma, np.array([0.5 + 0.5j]), np.array([1.0]))
    assert abs(ind[0] - want) <= 1e-13
    assert (ind[0] > 0.05) == (delta > 0)
    eig, _ = _gpu_vs_oracle(simlib, A, (0, 1, 0, 1), h0=1e-3)
    assert eig.size == 0
