"""GB300-native SIM-M: the multilevel spectral indicator method for all
eigenvalues of a sparse pencil A x = λ B x inside a region of the complex
plane, on one GPU.

The compute path lives in ``libsim.so`` (hand-written sm_103a CUDA behind the
C ABI declared in ``include/sim.h``); this package only marshals arguments to
it through ctypes.  Importing works without a GPU; every call into the library
requires the built ``libsim.so`` and raises if it is missing — there is no
CPU fallback.
"""
from ._binding import (  # noqa: F401
    SIM_FP64,
    SIM_MIXED,
    SimError,
    SimOptions,
    SimStats,
    Sim,
    Batch,
    eval_squares,
    lib,
    library_path,
    random_vectors,
    kernel_timing,
    kernel_stats,
    measure_fma_peak,
    launch_count,
    sim_default_options,
    run,
)
