"""Seeded synthetic inputs for SIM-M (pencils, regions, random vectors).

This module builds the matrices, search regions and random vectors that both
the CUDA path and the CPU oracle consume.  It holds none of SIM-M's own
arithmetic: no Krylov bases, no quadrature, no indicators.  Everything here is
deterministic given its seed.

Operators follow the workloads named for the method's benchmarks: constant
coefficient convection-diffusion  -Δu + b·∇u  on the unit square, discretised
with the 5-point central-difference stencil on an N×N interior grid
(h = 1/(N+1), Dirichlet boundary, lexicographic order with x fastest), optionally
with a diagonal B and appended Jordan blocks.
"""
from .pencils import (  # noqa: F401
    Csr,
    cd2d_csr,
    cd2d_eigenvalues,
    cdr_axes,
    cdr_csr,
    cdr_separable_eigenvalues,
    tridiag_toeplitz_csr,
    jordan_csr,
    pair_blocks_csr,
    block_diag_csr,
    diag_csr,
    identity_csr,
    dense_to_csr,
    complex_gaussian,
)
from .configs import config_small, config_pencil, config_jordan_small, config_cdr2d, config_cdr3d, config_batch, Workload  # noqa: F401
