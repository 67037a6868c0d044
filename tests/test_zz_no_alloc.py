"""sim_apply_shifted_noalloc: the shifted sparse apply for callers that must
not allocate device memory (their GPU memory belongs to another allocator, or
they cannot afford the synchronisation an allocation may cause).  It must give
the same y = (A - σB) x as sim_apply_shifted, call after call, with its
staging vectors in the library's static device array.

Collected last on purpose: run alone it checks the first-call set-up on a
fresh process; run after the other tests it checks that the shared static
array is reused correctly."""
import ctypes

import numpy as np
import pytest

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


def _apply(sim, s, fn, sigma, x):
    y = torch.empty_like(x)
    st = fn(s.h, float(np.real(sigma)), float(np.imag(sigma)), ctypes.c_void_p(x.data_ptr()),
            ctypes.c_void_p(y.data_ptr()))
    return st, y


def test_noalloc_apply_matches_allocating_apply_on_consecutive_calls(simlib):
    from workloads import cd2d_csr, diag_csr

    A = cd2d_csr(40, (1.0, 0.5))
    bd = np.random.default_rng(5).uniform(1.0, 2.0, A.n)
    s = simlib.Sim(A, diag_csr(bd))
    lib = simlib.lib()
    rng = np.random.default_rng(6)
    for sigma in (3000.0 + 0.2j, -15.5 + 4.0j):  # two calls in a row, different inputs
        x = torch.from_numpy(rng.standard_normal(A.n) + 1j * rng.standard_normal(A.n)).cuda()
        st_ref, y_ref = _apply(simlib, s, lib.sim_apply_shifted, sigma, x)
        st, y = _apply(simlib, s, lib.sim_apply_shifted_noalloc, sigma, x)
        assert st_ref == 0 and st == 0, lib.sim_last_error(s.h)
        ref = y_ref.cpu().numpy()
        got = y.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
        dense = (A.to_scipy() - sigma * diag_csr(bd).to_scipy()) @ x.cpu().numpy()
        assert np.max(np.abs(got - dense)) <= 1e-13 * np.max(np.abs(dense))
    s.close()


def test_noalloc_apply_leaves_free_device_memory_unchanged(simlib):
    """After the first call on the device (which loads the static array), a
    call must not change the device's free memory: it allocates nothing."""
    from workloads import cd2d_csr

    A = cd2d_csr(30, (1.0, 0.5))
    s = simlib.Sim(A, None)
    lib = simlib.lib()
    rng = np.random.default_rng(7)
    x = torch.from_numpy(rng.standard_normal(A.n) + 1j * rng.standard_normal(A.n)).cuda()
    y = torch.empty_like(x)
    args = (s.h, 100.0, 0.5, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    assert lib.sim_apply_shifted_noalloc(*args) == 0, lib.sim_last_error(s.h)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert lib.sim_apply_shifted_noalloc(*args) == 0, lib.sim_last_error(s.h)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    s.close()


def test_noalloc_apply_at_its_static_limit_matches_allocating_apply(simlib):
    from workloads import tridiag_toeplitz_csr

    n = 262144  # the largest n the static array holds
    T = tridiag_toeplitz_csr(n, -1.0 + 0.25j, 2.0, -1.0)
    s = simlib.Sim(T, None)
    lib = simlib.lib()
    rng = np.random.default_rng(8)
    x = torch.from_numpy(rng.standard_normal(n) + 1j * rng.standard_normal(n)).cuda()
    st_ref, y_ref = _apply(simlib, s, lib.sim_apply_shifted, 1.5 - 0.5j, x)
    st, y = _apply(simlib, s, lib.sim_apply_shifted_noalloc, 1.5 - 0.5j, x)
    assert st_ref == 0 and st == 0, lib.sim_last_error(s.h)
    ref = y_ref.cpu().numpy()
    assert np.max(np.abs(y.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))
    s.close()


def test_noalloc_apply_rejects_sizes_beyond_its_static_limit(simlib):
    from workloads import tridiag_toeplitz_csr

    n = 262144 + 1
    s = simlib.Sim(tridiag_toeplitz_csr(n, -1.0, 2.0, -1.0), None)
    lib = simlib.lib()
    x = torch.zeros(n, dtype=torch.complex128, device="cuda")
    st, _ = _apply(simlib, s, lib.sim_apply_shifted_noalloc, 0.5 + 0.5j, x)
    assert st == 7  # SIM_ERR_LIMIT
    assert b"262144" in lib.sim_last_error(s.h)
    s.close()
