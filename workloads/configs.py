"""Named synthetic workloads.

* ``config_small``  — 2-D convection–diffusion -Δu + (1, 0.5)·∇u, N = 30
  (n = 900), B = I, a search region holding exactly 50 closed-form
  eigenvalues with its vertical edges at midpoints between eigenvalues and
  Im range [-0.3, 0.7]; f complex Gaussian from seed 0.
* ``config_pencil`` — the same operator on a 200×200 grid (n = 40,000) with
  B = diag(uniform[1, 2]) from seed 1, plus a 64×64 block of sixteen 4×4
  Jordan blocks λI + νN (ν = 1e-7, B-block = I) appended at the end
  (n = 40,064); the region
  holds 500 eigenvalues of the convection–diffusion pencil (counted by
  Sylvester inertia, stored in ``regions.json``) and the 16 Jordan
  eigenvalues, each of algebraic multiplicity 4.
* ``config_jordan_small`` — a small pencil mixing a convection–diffusion
  block and Jordan blocks, for multiplicity tests that the oracle finishes in
  seconds.

These stand in for the paper's SuiteSparse matrices, which are not available.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field

import numpy as np

from .pencils import (
    Csr,
    block_diag_csr,
    cdr_axes,
    cdr_csr,
    cdr_separable_eigenvalues,
    cd2d_csr,
    cd2d_eigenvalues,
    complex_gaussian,
    diag_csr,
    jordan_csr,
)

_HERE = os.path.dirname(os.path.abspath(__file__))


@dataclass
class Workload:
    name: str
    A: Csr
    B: Csr | None          # None means B = I
    region: tuple           # (re_lo, re_hi, im_lo, im_hi)
    f: np.ndarray
    options: dict = field(default_factory=dict)
    expected_count: int | None = None   # Σ multiplicities inside R, from closed forms / inertia
    reference_eigs: np.ndarray | None = None  # closed-form eigenvalues inside R, when known
    reference_mult: np.ndarray | None = None
    separable: tuple | None = None  # (dims, (sub, diag, sup) per axis) of a separable principal part


def window_region(lam_sorted_real: np.ndarray, start: int, count: int, im=(-0.3, 0.7)):
    """Region whose real edges are midpoints around lam[start:start+count]."""
    lo = 0.5 * (lam_sorted_real[start - 1] + lam_sorted_real[start])
    hi = 0.5 * (lam_sorted_real[start + count - 1] + lam_sorted_real[start + count])
    return (float(lo), float(hi), float(im[0]), float(im[1]))


def max_gap_window(lr: np.ndarray, count: int, lo: int, hi: int) -> int:
    """Start index in [lo, hi) of the window of ``count`` consecutive sorted
    eigenvalues whose smallest gap (including the gaps to both outside
    neighbours) is largest; the first such window wins ties."""
    best, arg = -1.0, lo
    for s in range(max(lo, 1), min(hi, lr.size - count)):
        g = float(np.diff(lr[s - 1: s + count + 1]).min())
        if g > best:
            best, arg = g, s
    return arg


def config_small(seed: int = 0) -> Workload:
    N = 30
    A = cd2d_csr(N, (1.0, 0.5))
    lam = cd2d_eigenvalues(N, (1.0, 0.5))
    lr = np.sort(lam.real)
    start = max_gap_window(lr, 50, lr.size // 3, 2 * lr.size // 3)
    region = window_region(lr, start, 50)
    inside = lam[(lam.real > region[0]) & (lam.real < region[1])]
    return Workload(
        name="cd2d-30x30-I (n=900, 50 eigenvalues)",
        A=A, B=None, region=region, f=complex_gaussian(A.n, seed),
        options=dict(m=50, n0=4, delta0=0.05, eps=1e-8, h0=1e-6),
        expected_count=int(inside.size), reference_eigs=np.sort_complex(inside),
        reference_mult=np.ones(inside.size, dtype=np.int64),
    )


def _regions():
    with open(os.path.join(_HERE, "regions.json")) as fh:
        return json.load(fh)


def pencil_parts(N: int = 200, seed_b: int = 1):
    A = cd2d_csr(N, (1.0, 0.5))
    rng = np.random.default_rng(seed_b)
    bdiag = rng.uniform(1.0, 2.0, A.n)
    return A, bdiag


# Superdiagonal of the appended Jordan blocks.  Any ν != 0 gives the same
# Jordan structure (diag(1, ν, ν², ν³) scaling maps one to the other); a small ν
# keeps the rounding split of the defective eigenvalue, ~(ε||A|| ν³)^(1/4),
# far below h0.
JORDAN_SUP = 1e-7


def jordan_eigs(region, count: int = 16, im: float = 0.35):
    re_lo, re_hi = region[0], region[1]
    W = re_hi - re_lo
    t = np.arange(count)
    return re_lo + (t + 0.5) * W / count + 1j * im


def config_pencil(seed: int = 0, with_jordan: bool = True) -> Workload:
    reg = _regions()["pencil200"]
    region = tuple(reg["region"])
    A0, bdiag = pencil_parts(200, 1)
    if with_jordan:
        je = jordan_eigs(region)
        A = block_diag_csr(A0, jordan_csr(je, 4, JORDAN_SUP))
        B = diag_csr(np.concatenate([bdiag, np.ones(4 * je.size)]))
        count = reg["count"] + 4 * je.size
    else:
        A, B, je = A0, diag_csr(bdiag), np.zeros(0)
        count = reg["count"]
    return Workload(
        name="cd2d-200x200-diagB+jordan (n=%d)" % A.n,
        A=A, B=B, region=region, f=complex_gaussian(A.n, seed),
        options=dict(m=50, n0=4, delta0=0.05, eps=1e-8, h0=1e-6),
        expected_count=int(count),
    )


def config_jordan_small(seed: int = 0, sup: float = JORDAN_SUP) -> Workload:
    """n = 144 + 32: a 12×12 convection–diffusion block (B = I) and eight 4×4
    Jordan blocks placed inside a region around part of its spectrum."""
    N = 12
    A0 = cd2d_csr(N, (1.0, 0.5))
    lam = cd2d_eigenvalues(N, (1.0, 0.5))
    lr = np.sort(lam.real)
    start = 40
    region = window_region(lr, start, 30)
    je = jordan_eigs(region, count=8, im=0.35)
    A = block_diag_csr(A0, jordan_csr(je, 4, sup))
    inside = lam[(lam.real > region[0]) & (lam.real < region[1])]
    eigs = np.concatenate([inside, je])
    mult = np.concatenate([np.ones(inside.size, dtype=np.int64), np.full(je.size, 4)])
    order = np.lexsort((eigs.imag, eigs.real))
    return Workload(
        name="cd2d-12x12+jordan4x8 (n=176)",
        A=A, B=None, region=region, f=complex_gaussian(A.n, seed),
        options=dict(m=50, n0=4, delta0=0.05, eps=1e-8, h0=1e-6),
        expected_count=int(inside.size + 4 * je.size),
        reference_eigs=eigs[order], reference_mult=mult[order],
    )


# ---------------------------------------------------------------------------
# separable-principal-part workloads: 2-D and 3-D convection–diffusion–reaction
# ---------------------------------------------------------------------------
def _low_end_window(lam_real: np.ndarray, count: int, spread: float) -> tuple[int, float, float]:
    """Left edge below the smallest eigenvalue and a right edge in the first gap
    after `count` eigenvalues wide enough for a perturbation moving each
    eigenvalue by at most `spread` to the right; returns (count, lo, hi)."""
    lr = np.sort(lam_real)
    c = count
    while lr[c] - lr[c - 1] <= spread + 1.0:
        c += 1
    return c, float(lr[0] - 2.0), float(0.5 * (lr[c - 1] + spread + lr[c]))


def config_cdr2d(N: int = 500, count: int = 20, seed: int = 0) -> Workload:
    """2-D convection–diffusion–reaction -Δu + (1, 0.5)·∇u + c u on an N×N grid
    (n = N², 250,000 at N = 500), c_i ~ U[0,1] (seed 5), B = I: similar to a
    symmetric matrix with 0 <= c <= 1 added, so every eigenvalue is real and
    lies within [0, 1] to the right of one of the closed-form eigenvalues of
    the separable part.  The region spans the low end of the spectrum up to a
    gap, holding `count` or a few more eigenvalues, with Im range [-0.3, 0.7]."""
    beta = (1.0, 0.5)
    c = np.random.default_rng(5).uniform(0.0, 1.0, N * N)
    A = cdr_csr((N, N), beta, c)
    lam = cdr_separable_eigenvalues((N, N), beta)
    cnt, lo, hi = _low_end_window(lam.real, count, 1.0)
    return Workload(
        name="cdr2d-%dx%d reaction U[0,1] (n=%d, %d eigenvalues)" % (N, N, N * N, cnt),
        A=A, B=None, region=(lo, hi, -0.3, 0.7), f=complex_gaussian(A.n, seed),
        options=dict(m=50, n0=4, delta0=0.05, eps=1e-8, h0=1e-6),
        expected_count=cnt,
        separable=((N, N), cdr_axes((N, N), beta)),
    )


def config_cdr3d(N: int = 100, width: float = 140.0, seed: int = 0, at: float = 0.25) -> Workload:
    """3-D convection–diffusion–reaction -Δu + (1, 0.5, 0.25)·∇u + r u on an
    N×N×N grid (n = N³, 10⁶ at N = 100), r_i = sqrt(U) e^{2πiV} uniform in the
    unit disk (seed 4), B = I.  The region is `width` units of Re centred on the
    point a fraction `at` along the separable part's spectrum, Im [-1.3, 1.7]."""
    beta = (1.0, 0.5, 0.25)
    rng = np.random.default_rng(4)
    U, V = rng.uniform(size=N**3), rng.uniform(size=N**3)
    r = np.sqrt(U) * np.exp(2j * np.pi * V)
    A = cdr_csr((N, N, N), beta, r)
    lam = cdr_separable_eigenvalues((N, N, N), beta).real
    mid = float(lam.min() + at * (lam.max() - lam.min()))
    region = (mid - 0.5 * width, mid + 0.5 * width, -1.3, 1.7)
    return Workload(
        name="cdr3d-%d^3 complex reaction in the unit disk (n=%d), Re width %g" % (N, N**3, width),
        A=A, B=None, region=region, f=complex_gaussian(A.n, seed),
        options=dict(m=50, n0=4, delta0=0.05, eps=1e-8, h0=1e-6, init_side=1.0),
        separable=((N, N, N), cdr_axes((N, N, N), beta)),
    )


# ---------------------------------------------------------------------------
# batches of independent convection–diffusion pencils of uneven size
# ---------------------------------------------------------------------------
@dataclass
class BatchWorkload:
    name: str
    pencils: list          # Workload per pencil (B = I, separable principal part)
    expected_count: int    # Σ closed-form eigenvalues inside the regions


def config_batch(count: int = 64, seed: int = 3, n_lo: int = 45, n_span: int = 179, eig_lo: int = 20,
                 eig_hi: int = 300) -> BatchWorkload:
    """`count` pencils -Δu + β_p·∇u on N_p×N_p grids, N_p = n_lo + floor(n_span U_p),
    Péclet numbers Pe_p ~ U[0.1, 10] with β_p = Pe_p (1, 0.5)/||(1, 0.5)||, B = I
    (default_rng(seed)).  Each region is the window of c_p ~ U{eig_lo..eig_hi}
    consecutive closed-form eigenvalues (clipped to the middle third of the
    spectrum) with the largest smallest gap, Im [-0.3, 0.7]; f_p from seed p."""
    rng = np.random.default_rng(seed)
    Ns = n_lo + np.floor(n_span * rng.uniform(size=count)).astype(int)
    Pe = rng.uniform(0.1, 10.0, count)
    cs = rng.integers(eig_lo, eig_hi + 1, count)
    unit = np.array([1.0, 0.5]) / np.linalg.norm([1.0, 0.5])
    pencils, total = [], 0
    for p in range(count):
        N = int(Ns[p])
        beta = tuple(float(x) for x in Pe[p] * unit)
        lam = cd2d_eigenvalues(N, beta)
        lr = np.sort(lam.real)
        c = int(min(cs[p], lr.size // 3 - 2))
        start = max_gap_window(lr, c, lr.size // 3, 2 * lr.size // 3)
        region = window_region(lr, start, c)
        A = cdr_csr((N, N), beta)
        pencils.append(Workload(
            name="cd2d-%dx%d Pe=%.2f (%d eigenvalues)" % (N, N, Pe[p], c), A=A, B=None, region=region,
            f=complex_gaussian(A.n, p), options=dict(m=50, n0=4, delta0=0.05, eps=1e-8, h0=1e-6),
            expected_count=c, separable=((N, N), cdr_axes((N, N), beta))))
        total += c
    return BatchWorkload(name="%d convection-diffusion pencils, grids %d^2..%d^2, Pe U[0.1,10]" % (
        count, int(Ns.min()), int(Ns.max())), pencils=pencils, expected_count=total)
