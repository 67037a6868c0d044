"""Sparse test pencils in CSR form (int32 row pointers / column indices,
complex128 values) and the seeded complex Gaussian vector generator.

Only matrix *construction* lives here.  Closed-form spectra are provided for
input design (choosing a search region whose edges fall between eigenvalues)
and for tests; they are the textbook formulas for tridiagonal Toeplitz
matrices and their Kronecker sums.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Csr:
    """A square sparse matrix in CSR form.

    indptr  int32[n+1], indices int32[nnz] (sorted within each row),
    data    complex128[nnz].
    """

    n: int
    indptr: np.ndarray
    indices: np.ndarray
    data: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.n), dtype=np.complex128)
        for i in range(self.n):
            lo, hi = self.indptr[i], self.indptr[i + 1]
            out[i, self.indices[lo:hi]] += self.data[lo:hi]
        return out

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.n, self.n))


def _from_coo(n: int, rows, cols, vals) -> Csr:
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.complex128)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    # merge duplicates
    if rows.size:
        key = rows * n + cols
        uniq, start = np.unique(key, return_index=True)
        vals = np.add.reduceat(vals, start)
        rows = uniq // n
        cols = uniq % n
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return Csr(n, indptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.complex128))


def dense_to_csr(a: np.ndarray, drop_zeros: bool = True) -> Csr:
    a = np.asarray(a, dtype=np.complex128)
    n = a.shape[0]
    if drop_zeros:
        r, c = np.nonzero(a)
    else:
        r, c = np.indices(a.shape).reshape(2, -1)
    return _from_coo(n, r, c, a[r, c])


def identity_csr(n: int) -> Csr:
    i = np.arange(n)
    return _from_coo(n, i, i, np.ones(n))


def diag_csr(d) -> Csr:
    d = np.asarray(d, dtype=np.complex128)
    i = np.arange(d.size)
    return _from_coo(d.size, i, i, d)


def tridiag_toeplitz_csr(n: int, sub: complex, diag: complex, sup: complex) -> Csr:
    """Tridiagonal Toeplitz matrix with constant sub-, main and super-diagonal.

    Its eigenvalues are diag + 2*sqrt(sub*sup)*cos(k*pi/(n+1)), k = 1..n.
    """
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    vals = np.concatenate([np.full(n, diag), np.full(n - 1, sub), np.full(n - 1, sup)])
    return _from_coo(n, rows, cols, vals.astype(np.complex128))


def cd2d_csr(N: int, beta=(1.0, 0.5), reaction=None) -> Csr:
    """5-point central-difference discretisation of -Δu + beta·∇u (+ c u).

    Unit square, N×N interior nodes, h = 1/(N+1), Dirichlet boundary, unknown
    (ix, iy) at index iy*N + ix (x fastest).  ``reaction`` is an optional
    length-N*N array added to the diagonal.
    """
    h = 1.0 / (N + 1)
    b1, b2 = float(beta[0]), float(beta[1])
    n = N * N
    idx = np.arange(n)
    ix = idx % N
    iy = idx // N
    diag = np.full(n, 4.0 / h**2, dtype=np.complex128)
    if reaction is not None:
        diag = diag + np.asarray(reaction, dtype=np.complex128)
    rows = [idx]
    cols = [idx]
    vals = [diag]
    east = -1.0 / h**2 + b1 / (2 * h)
    west = -1.0 / h**2 - b1 / (2 * h)
    north = -1.0 / h**2 + b2 / (2 * h)
    south = -1.0 / h**2 - b2 / (2 * h)
    for mask, off, v in (
        (ix < N - 1, 1, east),
        (ix > 0, -1, west),
        (iy < N - 1, N, north),
        (iy > 0, -N, south),
    ):
        r = idx[mask]
        rows.append(r)
        cols.append(r + off)
        vals.append(np.full(r.size, v, dtype=np.complex128))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def cdr_axes(dims, beta):
    """(sub, diag, sup) of the 1-D factors tridiag(-1/h²-b/2h, 2/h², -1/h²+b/2h),
    h = 1/(N+1), one per axis: the separable part of :func:`cdr_csr`."""
    out = []
    for N, b in zip(dims, beta):
        h = 1.0 / (N + 1)
        out.append((-1.0 / h**2 - b / (2 * h), 2.0 / h**2, -1.0 / h**2 + b / (2 * h)))
    return np.array(out, dtype=np.complex128)


def cdr_csr(dims, beta, reaction=None) -> Csr:
    """Central-difference -Δu + beta·∇u + c u on the unit box with dims[d]
    interior nodes along axis d (1 to 3 axes), h_d = 1/(dims[d]+1), Dirichlet
    boundary, axis 0 fastest: the Kronecker sum of the 1-D factors of
    :func:`cdr_axes` plus diag(reaction)."""
    dims = [int(N) for N in dims]
    n = int(np.prod(dims))
    ax = cdr_axes(dims, beta)
    idx = np.arange(n)
    diag = np.zeros(n, dtype=np.complex128)
    rows, cols, vals = [], [], []
    stride = 1
    for d, N in enumerate(dims):
        sub, dg, sup = ax[d]
        i = (idx // stride) % N
        diag += dg
        for mask, off, v in ((i < N - 1, stride, sup), (i > 0, -stride, sub)):
            r = idx[mask]
            rows.append(r)
            cols.append(r + off)
            vals.append(np.full(r.size, v, dtype=np.complex128))
        stride *= N
    if reaction is not None:
        diag = diag + np.asarray(reaction, dtype=np.complex128)
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def cdr_separable_eigenvalues(dims, beta) -> np.ndarray:
    """Closed-form spectrum of the separable part of :func:`cdr_csr` (no
    reaction), sorted by (Re, Im)."""
    lam = np.zeros(1, dtype=np.complex128)
    for N, b in zip(dims, beta):
        lam = (lam[:, None] + cd1d_eigenvalues(int(N), float(b))[None, :]).ravel()
    return lam[np.lexsort((lam.imag, lam.real))]


def cd1d_eigenvalues(N: int, b: float) -> np.ndarray:
    """Eigenvalues of the 1-D factor tridiag(-1/h²-b/2h, 2/h², -1/h²+b/2h)."""
    h = 1.0 / (N + 1)
    k = np.arange(1, N + 1)
    prod = (1.0 / h**2 + b / (2 * h)) * (1.0 / h**2 - b / (2 * h))
    return 2.0 / h**2 + 2.0 * np.sqrt(prod + 0j) * np.cos(k * np.pi / (N + 1))


def cd2d_eigenvalues(N: int, beta=(1.0, 0.5)) -> np.ndarray:
    """Closed-form spectrum of :func:`cd2d_csr` (no reaction): the Kronecker
    sum of two tridiagonal Toeplitz matrices, sorted by (Re, Im)."""
    mx = cd1d_eigenvalues(N, float(beta[0]))
    my = cd1d_eigenvalues(N, float(beta[1]))
    lam = (mx[None, :] + my[:, None]).ravel()
    return lam[np.lexsort((lam.imag, lam.real))]


def jordan_csr(eigs, size: int = 4, sup: float = 1.0) -> Csr:
    """Block diagonal of Jordan blocks λI + sup·N (N: ones on the superdiagonal)."""
    eigs = np.asarray(eigs, dtype=np.complex128)
    n = eigs.size * size
    rows, cols, vals = [], [], []
    for t, lam in enumerate(eigs):
        base = t * size
        for i in range(size):
            rows.append(base + i)
            cols.append(base + i)
            vals.append(lam)
            if i + 1 < size:
                rows.append(base + i)
                cols.append(base + i + 1)
                vals.append(sup)
    return _from_coo(n, rows, cols, vals)


def pair_blocks_csr(alphas, betas) -> Csr:
    """Block diagonal of real 2×2 blocks [[a, b], [-b, a]] with eigenvalues a ± ib."""
    rows, cols, vals = [], [], []
    for t, (a, b) in enumerate(zip(alphas, betas)):
        i = 2 * t
        rows += [i, i, i + 1, i + 1]
        cols += [i, i + 1, i, i + 1]
        vals += [a, b, -b, a]
    return _from_coo(2 * len(alphas), rows, cols, vals)


def block_diag_csr(*mats: Csr) -> Csr:
    rows, cols, vals = [], [], []
    off = 0
    for m in mats:
        r = np.repeat(np.arange(m.n), np.diff(m.indptr))
        rows.append(r + off)
        cols.append(m.indices.astype(np.int64) + off)
        vals.append(m.data)
        off += m.n
    return _from_coo(off, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def complex_gaussian(n: int, seed: int) -> np.ndarray:
    """(N(0,1) + i N(0,1)) / sqrt(2) from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((2, n))
    return (z[0] + 1j * z[1]) / np.sqrt(2.0)
