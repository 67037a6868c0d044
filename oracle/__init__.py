"""CPU oracle for SIM-M — TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 NumPy/SciPy implementation of the multilevel spectral
indicator method (Huang, Sun, Yang), written step by step from the paper,
plus exact checkers (Sylvester inertia counts) and the Philox4x64-10 stream
the multiplicity step draws its random vectors from.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything in this package.  The CUDA product
path never does, and shares no code with it.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed-form spectra and indicators, Arnoldi invariants, the explicit residual,
dense QZ on small pencils, Jordan and Laplacian multiplicities, numpy's own
Philox stream, dense-eigensolver inertia counts).
"""
from .simm import Options, SimM, sim_m, Result  # noqa: F401
