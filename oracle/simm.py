"""Plain FP64 CPU SIM-M: the oracle the CUDA path is checked against.

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports this package; only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may run it.  It shares no code with the CUDA path.

Each function follows one step of SIM-M (Huang, Sun, Yang, "A Multilevel
Spectral Indicator Method for Eigenvalues of Large Non-Hermitian Matrices"):

* Cayley transform and Krylov subspace (Sec. 2, Eqs. IMxb, eq:5): the systems
  (A - zB)x = f become (I + (σ - z)M)x = b with M = (A - σB)^{-1}B and
  b = (A - σB)^{-1}f; one Krylov space K_m(M; b) serves every z.
* Arnoldi (Sec. 2, Eq. eq:arnoldi) — here with classical Gram–Schmidt applied
  twice (CGS2); inner solves with (A - σB) by a sparse LU (scipy ``splu``).
* Projected shifted solve (Eq. eq:many) and its residual (Eq. eq:error).
* Trapezoid quadrature of the spectral projection on the circle circumscribing
  a square (Sec. 2, Eqs. XLXf, IndicatorPf) and the memory-efficient indicator
  (Sec. 3.1, Eq. DeltaSm) with threshold δ0 (Def. 3.2).
* Multilevel subdivision (Sec. 3.3) and the SIM-M algorithm (Sec. 3.5).
* Multiplicity from the rank of [P f_1 … P f_k] (Sec. 3.4).
* Ritz refinement of the located eigenvalues from the eigenvalues of H_m
  (Sec. 3.2, Eq. zjHm: H_m = P D P^{-1}; an eigenvalue d of H_m is a Ritz value
  of M = (A - σB)^{-1}B, and λ = σ + 1/d).

Readings of points the paper leaves open are fixed in ``Options`` and in the
docstrings below (node angles, weight normalisation, residual normalisation,
initial tiling, shift rounds, merge and multiplicity details).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .philox import random_vectors

SQRT1_2 = 0.70710678118654752440  # 1/sqrt(2): circumradius of a unit square


@dataclass
class Options:
    """SIM-M parameters (Sec. 3.5 inputs) plus the readings this oracle fixes."""

    m: int = 50            # Krylov dimension (Sec. 3.5: m = 50)
    n0: int = 4            # coarse rule size; the fine rule has 2*n0 nodes (Sec. 3.1)
    delta0: float = 0.05   # indicator threshold δ0 = 1/20 (Sec. 3.1)
    eps: float = 1e-8      # residual tolerance ε (≡ ε0 of Def. 3.1)
    h0: float = 1e-6       # precision
    init_side: float = 0.0  # side s1 of the initial squares; 0 => min(W, H)
    shift_sep: float = 4.0  # minimum separation, in units of s1, of shifts made in one round
    max_shift_rounds: int = 16
    breakdown_tol: float = 1e-14
    merge_radius: float = 0.0
    mult_k: int = 8
    mult_kmax: int = 64
    mult_tol: float = 1e-6
    mult_nodes: int = 16
    mult_seed: int = 0x5EED
    residual_scale: str = "solution"  # "solution": ρ relative to ||y|| = ||x_m||; "beta": relative to β = ||b||
    max_squares: int = 4_000_000    # a level with more squares than this is an error
    mult_reorth: int = 0            # multiplicity spaces: 0 one Gram-Schmidt pass (as printed), 1 CGS2
    new_shifts_in_levels: int = 0   # 1: squares no shift resolves get new shifts at their centres (step 3's rounds
                                    # repeated at each level); 0: shifts only at initialisation, as printed


# ---------------------------------------------------------------------------
# Shift-invariant Krylov space of M = (A - σB)^{-1} B   (Sec. 2)
# ---------------------------------------------------------------------------
@dataclass
class KrylovSpace:
    sigma: complex
    H: np.ndarray          # (m_eff+1) × m_eff upper Hessenberg; H[m_eff, m_eff-1] = h_{m+1,m}
    beta: float            # ||b||_2, b = (A - σB)^{-1} f
    m_eff: int             # < m after a breakdown (h_{j+1,j} = 0)
    V: np.ndarray | None = None  # n × (m_eff+1) orthonormal basis (only if requested)


def shifted_factor(A, B, sigma):
    """Sparse LU of (A - σB); the inner solver of this oracle."""
    K = (A - sigma * B).tocsc()
    return spla.splu(K)


def cayley_arnoldi(A, B, sigma, f, m, breakdown_tol=1e-14, keep_basis=False, lu=None, passes=2):
    """Arnoldi for M = (A - σB)^{-1}B started from b = (A - σB)^{-1}f.

    Sec. 2: v_1 = b/||b||, then for j = 1..m: w = M v_j, h_ij = (w, v_i),
    w -= Σ h_ij v_i, h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}; stop if
    h_{j+1,j} = 0.  The projection is applied `passes` times (2: CGS2, the
    default; 1: the single pass as printed) and the coefficients summed.
    "Zero" is h_{j+1,j} <= breakdown_tol * ||H_{1:j+1,1:j}||_F.
    """
    n = A.shape[0]
    if lu is None:
        lu = shifted_factor(A, B, sigma)
    b = lu.solve(np.asarray(f, dtype=np.complex128))
    beta = float(np.linalg.norm(b))
    if not beta > 0:
        raise ValueError("b = (A - σB)^{-1} f is zero")
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    V[:, 0] = b / beta
    m_eff = m
    for j in range(m):
        w = lu.solve(B @ V[:, j])
        Vj = V[:, : j + 1]
        h = np.zeros(j + 1, dtype=np.complex128)
        for _ in range(passes):
            hp = Vj.conj().T @ w
            w = w - Vj @ hp
            h = h + hp
        H[: j + 1, j] = h
        hn = float(np.linalg.norm(w))
        if hn <= breakdown_tol * float(np.linalg.norm(H[: j + 1, : j + 1])):
            m_eff = j + 1
            H[j + 1, j] = 0.0
            break
        H[j + 1, j] = hn
        V[:, j + 1] = w / hn
    Hk = H[: m_eff + 1, :m_eff].copy()
    return KrylovSpace(sigma=complex(sigma), H=Hk, beta=beta, m_eff=m_eff,
                       V=V[:, : m_eff + 1].copy() if keep_basis else None)


# ---------------------------------------------------------------------------
# Projected shifted solves and residuals   (Eqs. eq:many, eq:error)
# ---------------------------------------------------------------------------
def projected_solve(ks: KrylovSpace, z, scale: str = "solution"):
    """y = β (I + (σ - z)H_m)^{-1} e_1 for an array of points z (Eq. eq:y).

    Returns (y, rho): y has shape z.shape + (m_eff,), and rho is the residual of
    Eq. eq:error, |σ - z| h_{m+1,m} |e_m^T y|, divided by β = ||b|| (scale
    "beta", the residual relative to the right-hand side) or by ||y||_2 (scale
    "solution"; since V_m is orthonormal ||y|| = ||x_m||, so this is the
    residual relative to the size of the computed solution).
    """
    z = np.asarray(z, dtype=np.complex128)
    m = ks.m_eff
    Hm = ks.H[:m, :m]
    hlast = float(abs(ks.H[m, m - 1]))
    alpha = ks.sigma - z
    T = np.eye(m, dtype=np.complex128) + alpha[..., None, None] * Hm
    rhs = np.zeros(z.shape + (m,), dtype=np.complex128)
    rhs[..., 0] = ks.beta
    y = np.linalg.solve(T, rhs[..., None])[..., 0]
    ynorm = np.linalg.norm(y, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.abs(alpha) * hlast * np.abs(y[..., m - 1]) / (ynorm if scale == "solution" else ks.beta)
    rho = np.where(np.isfinite(rho), rho, np.inf)
    return y, rho


def eig_decomposition(ks: KrylovSpace):
    """Sec. 3.2, Eq. zjHm: H_m = P D P^{-1}.  Returns the eigenvalues d, the
    eigenvector matrix P, c_1 = P^{-1} e_1 and r_m = e_m^T P (the last row)."""
    m = ks.m_eff
    d, P = np.linalg.eig(ks.H[:m, :m])
    e1 = np.zeros(m, dtype=np.complex128)
    e1[0] = 1.0
    c1 = np.linalg.solve(P, e1)
    return d, P, c1, P[m - 1, :].copy()


def screened_last_entry(ks: KrylovSpace, z, dec=None):
    """Sec. 3.2, Eq. rmLc1: e_m^T y_j = β r_m (I + (σ - z_j)D)^{-1} c_1, O(m) per
    point z_j once H_m's eigendecomposition is known (exact for a
    diagonalisable H_m; its rounding grows with the condition of P).  Returns
    e_m^T y for each z and the β-relative residual |σ - z| h_{m+1,m} |e_m^T y| / β
    of Eq. eq:error."""
    d, P, c1, rm = dec if dec is not None else eig_decomposition(ks)
    z = np.asarray(z, dtype=np.complex128)
    alpha = ks.sigma - z
    ym = ks.beta * np.sum(rm * c1 / (1.0 + alpha[..., None] * d), axis=-1)
    hlast = float(abs(ks.H[ks.m_eff, ks.m_eff - 1]))
    return ym, np.abs(alpha) * hlast * np.abs(ym) / ks.beta


# ---------------------------------------------------------------------------
# Quadrature on the circle circumscribing a square, and the indicator
# ---------------------------------------------------------------------------
def node_offsets(s):
    """Offsets z_j - c of the 8 nodes on the circle circumscribing a square of
    side s: radius r = s/sqrt(2), angle 2πj/8.  Even j: ±r, ±ir; odd j: the
    square's corners (±s/2)(1 ± i).  Shape (..., 8)."""
    s = np.asarray(s, dtype=np.float64)
    r = s * SQRT1_2
    hs = 0.5 * s
    re = np.stack([r, hs, 0 * s, -hs, -r, -hs, 0 * s, hs], axis=-1)
    im = np.stack([0 * s, hs, r, hs, 0 * s, -hs, -r, -hs], axis=-1)
    return re + 1j * im


def indicator_from_y(y, offsets):
    """Eq. DeltaSm: Ĩ = ||Σ_{j<8} w_j y_j|| / ||Σ_{j even} w'_j y_j||.

    The quadrature weight of the N-point trapezoid rule for (1/2πi)∮ g dz on a
    circle centred at c is (z_j - c)/N, so w_j = (z_j - c)/8 on the fine rule
    and w'_j = (z_j - c)/4 on the coarse rule (the even nodes).  Ĩ = 0 when
    both sums vanish, +inf when only the coarse sum does.
    """
    Y8 = np.einsum("...j,...jk->...k", offsets / 8.0, y)
    Y4 = np.einsum("...j,...jk->...k", offsets[..., 0::2] / 4.0, y[..., 0::2, :])
    n8 = np.linalg.norm(Y8, axis=-1)
    n4 = np.linalg.norm(Y4, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        ind = np.where(n4 > 0, n8 / np.where(n4 > 0, n4, 1.0), np.where(n8 > 0, np.inf, 0.0))
    return ind


def evaluate_squares(ks: KrylovSpace, centers, sides, scale: str = "solution"):
    """Nodes, projected solves, residuals and indicator of squares w.r.t. one shift.

    Returns (indicator, resolvable) arrays of the squares' shape.  Resolvable
    (Def. 3.1) means rho <= ε at all 8 nodes; this needs ``eps`` so it is
    applied by the caller — here rho_max is returned instead.
    """
    centers = np.asarray(centers, dtype=np.complex128).ravel()
    sides = np.broadcast_to(np.asarray(sides, dtype=np.float64), centers.shape)
    ind = np.zeros(centers.shape)
    rmax = np.zeros(centers.shape)
    for a in range(0, centers.size, 512):  # bounded memory: 512 squares at a time
        off = node_offsets(sides[a:a + 512])
        z = centers[a:a + 512, None] + off
        y, rho = projected_solve(ks, z, scale)
        ind[a:a + 512] = indicator_from_y(y, off)
        rmax[a:a + 512] = rho.max(axis=-1)
    return ind, rmax


# ---------------------------------------------------------------------------
# Square lattice.  Level-k squares have side s_k = s1 / 2^(k-1) and integer
# lattice coordinates (ix, iy); centre = (re_lo + (ix + 1/2)s_k, im_lo + (iy + 1/2)s_k).
# ---------------------------------------------------------------------------
def square_centers(re_lo, im_lo, s, ix, iy):
    ix = np.asarray(ix, dtype=np.float64)
    iy = np.asarray(iy, dtype=np.float64)
    return (re_lo + (ix + 0.5) * s) + 1j * (im_lo + (iy + 0.5) * s)


def initial_tiling(region, s1):
    """Tile the bounding box of R with squares of side s1 from its lower-left
    corner: ceil(W/s1) columns by ceil(H/s1) rows, row-major (Im outer)."""
    re_lo, re_hi, im_lo, im_hi = region
    cols = max(1, int(math.ceil((re_hi - re_lo) / s1 - 1e-12)))
    rows = max(1, int(math.ceil((im_hi - im_lo) / s1 - 1e-12)))
    iy, ix = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    return ix.ravel().astype(np.int64), iy.ravel().astype(np.int64)


def num_levels(s1, h0):
    """K such that s_K = s1/2^(K-1) <= h0 (the level whose squares reach h0)."""
    return int(math.ceil(math.log2(s1 / h0))) + 1 if s1 > h0 else 1


# ---------------------------------------------------------------------------
# SIM-M driver
# ---------------------------------------------------------------------------
@dataclass
class Result:
    eigenvalues: np.ndarray            # cluster estimates inside R, sorted by (Re, Im)
    multiplicities: np.ndarray | None  # one per eigenvalue (Sec. 3.4)
    cluster_shift: np.ndarray          # resolving shift id per eigenvalue
    cluster_size: np.ndarray           # final squares per eigenvalue
    cluster_flagged: np.ndarray        # members left unresolvable (warnings, step 6)
    shifts: list = field(default_factory=list)
    level_counts: list = field(default_factory=list)   # squares evaluated per level
    final_ix: np.ndarray | None = None
    final_iy: np.ndarray | None = None
    final_shift: np.ndarray | None = None
    final_flag: np.ndarray | None = None
    s_final: float = 0.0
    n_inner_solves: int = 0


class SimM:
    """SIM-M(A, B, R, f, h0, ε, δ0, m, n0) of Sec. 3.5, one step per method."""

    def __init__(self, A, B, opts: Options | None = None):
        self.A = sp.csr_matrix(A, dtype=np.complex128)
        n = self.A.shape[0]
        self.B = sp.identity(n, dtype=np.complex128, format="csr") if B is None else sp.csr_matrix(B, dtype=np.complex128)
        self.o = opts or Options()
        self.n = n
        self.spaces: list[KrylovSpace] = []
        self._lu = []
        self.n_inner_solves = 0

    # -- Krylov spaces -------------------------------------------------------
    def add_shift(self, sigma, f):
        lu = shifted_factor(self.A, self.B, sigma)
        ks = cayley_arnoldi(self.A, self.B, sigma, f, self.o.m, self.o.breakdown_tol, lu=lu)
        self.n_inner_solves += 1 + ks.m_eff
        self.spaces.append(ks)
        self._lu.append(lu)
        return len(self.spaces) - 1

    def shift_order(self, c):
        """Existing shifts ordered by |σ - c|, ties by shift id."""
        d = np.array([abs(ks.sigma - c) for ks in self.spaces])
        return list(np.lexsort((np.arange(d.size), d)))

    def resolve(self, centers, sides, shift_ids, try_all=True):
        """Evaluate squares with their shift; unresolvable ones try the other
        shifts nearest-first and move to the first that resolves them.

        Returns (indicator, resolvable, shift_ids)."""
        centers = np.asarray(centers)
        sides = np.broadcast_to(np.asarray(sides, dtype=np.float64), centers.shape)
        ind = np.zeros(centers.shape)
        res = np.zeros(centers.shape, dtype=bool)
        sid = np.array(shift_ids, dtype=np.int64)
        for s in np.unique(sid):
            sel = np.nonzero(sid == s)[0]
            i, r = evaluate_squares(self.spaces[s], centers[sel], sides[sel], self.o.residual_scale)
            ind[sel] = i
            res[sel] = r <= self.o.eps
        if try_all and len(self.spaces) > 1:
            for q in np.nonzero(~res)[0]:
                for s in self.shift_order(centers[q]):
                    if s == sid[q]:
                        continue
                    i, r = evaluate_squares(self.spaces[s], centers[q:q + 1], sides[q:q + 1], self.o.residual_scale)
                    if r[0] <= self.o.eps:
                        ind[q], res[q], sid[q] = i[0], True, s
                        break
        return ind, res, sid

    # -- Sec. 3.5 steps 1-3: first shift, initial squares, shift association --
    def set_region(self, region, f):
        o = self.o
        re_lo, re_hi, im_lo, im_hi = region
        self.region = region
        W, Hh = re_hi - re_lo, im_hi - im_lo
        self.s1 = o.init_side if o.init_side > 0 else min(W, Hh)
        self.f = np.asarray(f, dtype=np.complex128)
        ix, iy = initial_tiling(region, self.s1)
        c = square_centers(re_lo, im_lo, self.s1, ix, iy)
        # step 1: the centre of R is the first shift
        self.add_shift(complex(0.5 * (re_lo + re_hi), 0.5 * (im_lo + im_hi)), self.f)
        sid = np.zeros(ix.size, dtype=np.int64)
        resolved = np.zeros(ix.size, dtype=bool)
        # step 3 in rounds: test every unresolved square against every shift
        # (nearest first); then pick new shift centres among the squares still
        # unresolved, walking them in row-major order and keeping a square if it
        # lies at least D_r from every square kept in this round, where
        # D_r = max(shift_sep*s1, ρ) and ρ is the distance from the first shift
        # to the nearest initial square it does not resolve.
        sep = None
        for _ in range(o.max_shift_rounds):
            todo = np.nonzero(~resolved)[0]
            for q in todo:
                for s in self.shift_order(c[q]):
                    _, r = evaluate_squares(self.spaces[s], c[q:q + 1], np.array([self.s1]), o.residual_scale)
                    if r[0] <= o.eps:
                        resolved[q], sid[q] = True, s
                        break
            todo = np.nonzero(~resolved)[0]
            if todo.size == 0:
                break
            if sep is None:
                rho = float(np.min(np.abs(c[todo] - self.spaces[0].sigma)))
                sep = max(o.shift_sep * self.s1, rho)
            picked = []
            for q in todo:
                if all(abs(c[q] - c[p]) >= sep for p in picked):
                    picked.append(q)
            for q in picked:
                s = self.add_shift(c[q], self.f)
                sid[q] = s
        self.init_ix, self.init_iy, self.init_sid = ix, iy, sid
        self.K = num_levels(self.s1, o.h0)

    # -- Sec. 3.5 steps 4-5: the level loop (Sec. 3.3) ------------------------
    def solve_levels(self):
        o = self.o
        re_lo, _, im_lo, _ = self.region
        ix, iy, sid = self.init_ix, self.init_iy, self.init_sid
        self.level_counts = []
        for k in range(1, self.K + 1):
            s = self.s1 / 2.0 ** (k - 1)
            c = square_centers(re_lo, im_lo, s, ix, iy)
            ind, res, sid = self.resolve(c, s, sid)
            if o.new_shifts_in_levels:
                # step 3's rounds at this level: new Krylov spaces at the centres of
                # unresolved squares (list order, at least shift_sep·s apart), then
                # every square of the level evaluated again
                for _ in range(o.max_shift_rounds):
                    un = np.nonzero(~res)[0]
                    if un.size == 0:
                        break
                    picked = []
                    for q in un:
                        if all(abs(c[q] - c[p]) >= o.shift_sep * s for p in picked):
                            picked.append(q)
                    for q in picked:
                        self.add_shift(c[q], self.f)
                    ind, res, sid = self.resolve(c, s, sid)
            # resolvable: mark iff Ĩ > δ0; unresolvable: mark and flag (step 5)
            mark = np.where(res, ind > o.delta0, True)
            flag = ~res
            self.level_counts.append(int(ix.size))
            if k == self.K:
                keep = np.nonzero(mark)[0]
                self.final = (ix[keep], iy[keep], sid[keep], flag[keep], s)
                break
            keep = np.nonzero(mark)[0]
            # children SW, SE, NW, NE, in parent order
            dx = np.array([0, 1, 0, 1])
            dy = np.array([0, 0, 1, 1])
            if 4 * keep.size > o.max_squares:
                raise RuntimeError("level %d would hold %d squares (> max_squares)" % (k + 1, 4 * keep.size))
            ix = (2 * ix[keep][:, None] + dx).ravel()
            iy = (2 * iy[keep][:, None] + dy).ravel()
            sid = np.repeat(sid[keep], 4)
        return self.final

    # -- Sec. 3.5 step 6: merge ------------------------------------------------
    def merge(self):
        """8-connected components of the final squares (edge or corner
        contact); estimate = mean of member centres; components whose estimates
        are closer than merge_radius are joined; keep estimates inside closed R;
        sort by (Re, Im)."""
        o = self.o
        fix, fiy, fsid, fflag, s = self.final
        re_lo, re_hi, im_lo, im_hi = self.region
        nsq = fix.size
        parent = np.arange(nsq)

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        def union(a, b):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)

        pos = {(int(x), int(y)): i for i, (x, y) in enumerate(zip(fix, fiy))}
        for i in range(nsq):
            for ddx in (-1, 0, 1):
                for ddy in (-1, 0, 1):
                    j = pos.get((int(fix[i]) + ddx, int(fiy[i]) + ddy))
                    if j is not None:
                        union(i, j)
        centers = square_centers(re_lo, im_lo, s, fix, fiy)

        def components():
            roots = np.array([find(i) for i in range(nsq)], dtype=np.int64)
            labels, inv = np.unique(roots, return_inverse=True)
            est = np.zeros(labels.size, dtype=np.complex128)
            np.add.at(est, inv, centers)
            cnt = np.bincount(inv, minlength=labels.size)
            return labels, inv, est / cnt, cnt

        labels, inv, est, cnt = components()
        if o.merge_radius > 0 and labels.size > 1:
            for a in range(labels.size):
                for b in range(a + 1, labels.size):
                    if abs(est[a] - est[b]) < o.merge_radius:
                        union(labels[a], labels[b])
            labels, inv, est, cnt = components()
        inside = (est.real >= re_lo) & (est.real <= re_hi) & (est.imag >= im_lo) & (est.imag <= im_hi)
        # resolving shift of a cluster: that of its first member (list order)
        first = np.full(labels.size, nsq, dtype=np.int64)
        np.minimum.at(first, inv, np.arange(nsq))
        flagged = np.zeros(labels.size, dtype=np.int64)
        np.add.at(flagged, inv, fflag.astype(np.int64))
        # circumradius of each cluster: farthest member corner from the estimate
        far = np.abs(centers - est[inv]) + s * SQRT1_2
        rad = np.zeros(labels.size)
        np.maximum.at(rad, inv, far)
        keep = np.nonzero(inside)[0]
        order = keep[np.lexsort((est[keep].imag, est[keep].real))]
        self.clusters = dict(
            estimate=est[order], size=cnt[order], shift=fsid[first[order]],
            flagged=flagged[order], radius=rad[order],
        )
        return self.clusters

    # -- Sec. 3.2: Ritz refinement of the located eigenvalues -----------------
    def refine(self):
        """For each cluster: the Ritz values d_i = eig(H_m) of its resolving
        shift's Krylov space (Sec. 3.2, Eq. zjHm), mapped back by λ_i = σ + 1/d_i
        (the Cayley transform M = (A - σB)^{-1}B has eigenvalues 1/(λ - σ)).
        The λ_i nearest the cluster estimate replaces it if it lies within
        2·max(cluster radius, h0) of it (the multiplicity circle's radius);
        otherwise the estimate stays.  Returns (values, refined flags)."""
        o = self.o
        cl = self.clusters
        est = cl["estimate"]
        out = est.copy()
        flag = np.zeros(est.size, dtype=bool)
        for c in range(est.size):
            ks = self.spaces[cl["shift"][c]]
            d = np.linalg.eigvals(ks.H[: ks.m_eff, : ks.m_eff])
            d = d[d != 0]
            lam = ks.sigma + 1.0 / d
            i = int(np.argmin(np.abs(lam - est[c])))
            if abs(lam[i] - est[c]) <= 2.0 * max(cl["radius"][c], o.h0):
                out[c], flag[c] = lam[i], True
        return out, flag

    def projection(self, c):
        """P f for cluster c: the trapezoid rule (Sec. 2, Eq. XLXf) on the
        mult_nodes-node circle of radius 2·max(cluster radius, h0) around its
        estimate, applied to the region's vector f through the Krylov space of
        the resolving shift (rebuilt with its basis V):
        P f ≈ V Σ_j ((z_j - c)/N) y_j.  For a simple eigenvalue this is an
        eigenvector (Remark 3.5)."""
        o = self.o
        cl = self.clusters
        s = cl["shift"][c]
        ks = cayley_arnoldi(self.A, self.B, self.spaces[s].sigma, self.f, o.m, o.breakdown_tol, keep_basis=True,
                            lu=self._lu[s])
        unit = np.exp(2j * np.pi * np.arange(o.mult_nodes) / o.mult_nodes)
        off = 2.0 * max(cl["radius"][c], o.h0) * unit
        y, _ = projected_solve(ks, cl["estimate"][c] + off)
        u = (off / unit.size) @ y
        return ks.V[:, : ks.m_eff] @ u

    # -- Sec. 3.4: multiplicities ---------------------------------------------
    def multiplicity(self):
        """For each shift that resolves clusters: k random vectors f_i, the k
        Krylov spaces K_m^σ(M; b_i), P f_i on a 16-node circle around each
        cluster estimate of radius 2*max(radius, h0), and the number of singular
        values of [P f_1 … P f_k] above mult_tol times the largest.  k doubles
        while the rank equals k, up to mult_kmax."""
        o = self.o
        cl = self.clusters
        nclu = cl["estimate"].size
        mult = np.zeros(nclu, dtype=np.int64)
        Nq = o.mult_nodes
        ang = 2.0 * np.pi * np.arange(Nq) / Nq
        unit = np.cos(ang) + 1j * np.sin(ang)
        for s in np.unique(cl["shift"]):
            members = np.nonzero(cl["shift"] == s)[0]
            k = o.mult_k
            pending = members
            while pending.size:
                F = random_vectors(o.mult_seed, self.n, k)
                ranks = self._rank_for(s, F, pending, unit)
                done = (ranks < k) | (k >= o.mult_kmax)
                mult[pending[done]] = ranks[done]
                pending = pending[~done]
                k = min(2 * k, o.mult_kmax)
        self.clusters["multiplicity"] = mult
        return mult

    def _rank_for(self, s, F, members, unit):
        o = self.o
        cl = self.clusters
        sigma = self.spaces[s].sigma
        lu = self._lu[s]
        k = F.shape[1]
        Pf = np.zeros((members.size, self.n, k), dtype=np.complex128)
        for i in range(k):
            ks = cayley_arnoldi(self.A, self.B, sigma, F[:, i], o.m, o.breakdown_tol, keep_basis=True, lu=lu,
                                passes=2 if o.mult_reorth else 1)
            self.n_inner_solves += 1 + ks.m_eff
            for q, c in enumerate(members):
                rc = 2.0 * max(cl["radius"][c], o.h0)
                off = rc * unit
                y, _ = projected_solve(ks, cl["estimate"][c] + off)
                u = (off / unit.size) @ y
                Pf[q, :, i] = ks.V[:, : ks.m_eff] @ u
        ranks = np.zeros(members.size, dtype=np.int64)
        for q in range(members.size):
            sv = np.linalg.svd(Pf[q], compute_uv=False)
            ranks[q] = int(np.sum(sv > o.mult_tol * sv[0])) if sv[0] > 0 else 0
        return ranks

    def run(self, region, f, multiplicity=True) -> Result:
        self.set_region(region, f)
        self.solve_levels()
        cl = self.merge()
        mult = self.multiplicity() if multiplicity else None
        fix, fiy, fsid, fflag, s = self.final
        return Result(
            eigenvalues=cl["estimate"], multiplicities=mult, cluster_shift=cl["shift"],
            cluster_size=cl["size"], cluster_flagged=cl["flagged"],
            shifts=[ks.sigma for ks in self.spaces], level_counts=self.level_counts,
            final_ix=fix, final_iy=fiy, final_shift=fsid, final_flag=fflag, s_final=s,
            n_inner_solves=self.n_inner_solves,
        )


def sim_m(A, B, region, f, opts: Options | None = None, multiplicity=True) -> Result:
    """SIM-M(A, B, R, f, h0, ε, δ0, m, n0) (Sec. 3.5)."""
    return SimM(A, B, opts).run(region, f, multiplicity=multiplicity)
