"""ctypes binding of libsim.so.  Argument marshalling only: every step of
SIM-M runs in the library's CUDA kernels.  Names follow the C ABI
(``include/sim.h``)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "libsim.so")

SIM_FP64 = 0
SIM_MIXED = 1

STATUS = {0: "SIM_OK", 1: "SIM_ERR_INVALID_ARG", 2: "SIM_ERR_BAD_STATE", 3: "SIM_ERR_CUDA", 4: "SIM_ERR_OOM",
          5: "SIM_ERR_NOT_CONVERGED", 6: "SIM_ERR_CAPACITY", 7: "SIM_ERR_LIMIT"}


class SimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class SimCsr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p),
                ("values", C.c_void_p), ("on_device", C.c_int32)]


class SimOptions(C.Structure):
    _fields_ = [
        ("m", C.c_int32), ("n0", C.c_int32), ("delta0", C.c_double), ("eps", C.c_double), ("h0", C.c_double),
        ("init_side", C.c_double), ("shift_sep", C.c_double), ("max_shift_rounds", C.c_int32),
        ("max_shifts", C.c_int32), ("breakdown_tol", C.c_double), ("merge_radius", C.c_double),
        ("mult_k", C.c_int32), ("mult_kmax", C.c_int32), ("mult_tol", C.c_double), ("mult_nodes", C.c_int32),
        ("mult_seed", C.c_uint64), ("residual_scale", C.c_int32), ("max_squares", C.c_int64),
        ("precision", C.c_int32), ("inner_tol", C.c_double), ("inner_restart", C.c_int32),
        ("inner_max_iter", C.c_int32), ("mult_inner_tol", C.c_double), ("mult_reorth", C.c_int32),
        ("new_shifts_in_levels", C.c_int32), ("level_solver", C.c_int32), ("separable_tensor_cores", C.c_int32),
    ]


class SimStats(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("nnz_A", C.c_int64), ("nnz_B", C.c_int64), ("block_size", C.c_int32),
        ("num_blocks", C.c_int32), ("num_shifts", C.c_int32), ("levels_total", C.c_int32),
        ("levels_done", C.c_int32), ("squares_evaluated", C.c_int64), ("projected_solves", C.c_int64),
        ("inner_solves", C.c_int64), ("gmres_iterations", C.c_int64), ("max_gmres_iterations", C.c_int32),
        ("unresolvable_final", C.c_int64), ("final_squares", C.c_int64), ("clusters", C.c_int64),
        ("max_inner_residual", C.c_double), ("t_factor_ms", C.c_double), ("t_krylov_ms", C.c_double),
        ("t_levels_ms", C.c_double), ("t_merge_ms", C.c_double), ("t_mult_ms", C.c_double),
        ("loose_inner_solves", C.c_int64), ("unresolvable_last_level", C.c_int64), ("shift_retries", C.c_int64),
        ("direct_level_evaluations", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

EXPORTS = [
    "sim_default_options", "sim_create", "sim_set_region", "sim_solve_level", "sim_eigenvalues",
    "sim_multiplicity", "sim_refine", "sim_projection", "sim_stats", "sim_last_error", "sim_destroy", "sim_shift_count", "sim_get_shift",
    "sim_eval_squares", "sim_apply_shifted", "sim_shifted_solve", "sim_random_vectors",
    "sim_kernel_timing", "sim_kernel_stats", "sim_launch_count", "sim_apply_shifted_noalloc",
    "sim_set_separable", "sim_projection_norm", "sim_projection_norm_grad", "sim_eigenvalue_grad",
    "sim_update_values", "sim_measure_fma_peak",
    "sim_batch_create", "sim_batch_set_separable", "sim_batch_set_regions", "sim_batch_solve_level",
    "sim_batch_eigenvalues", "sim_batch_multiplicity", "sim_batch_handle", "sim_batch_last_error",
    "sim_batch_destroy", "sim_residual_screen",
]


def lib():
    """Load libsim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(library_path):
        raise RuntimeError("libsim.so is not built (run __graft_entry__.build()); SIM-M has no CPU fallback")
    L = C.CDLL(library_path)
    vp, i32, i64, u64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
    L.sim_default_options.argtypes = [C.POINTER(SimOptions)]
    L.sim_default_options.restype = None
    L.sim_create.argtypes = [C.POINTER(SimCsr), C.POINTER(SimCsr), C.POINTER(SimOptions), vp, C.POINTER(vp)]
    L.sim_set_region.argtypes = [vp, dbl, dbl, dbl, dbl, vp, i32, u64]
    L.sim_set_separable.argtypes = [vp, i32, vp, vp]
    L.sim_projection_norm.argtypes = [vp, dbl, dbl, dbl, i32, vp, i32, i32, C.POINTER(dbl)]
    L.sim_projection_norm_grad.argtypes = [vp, vp, vp, i32]
    L.sim_eigenvalue_grad.argtypes = [vp, dbl, dbl, dbl, i32, u64, vp, vp, vp, i32]
    L.sim_update_values.argtypes = [vp, vp, vp, i32]
    L.sim_measure_fma_peak.argtypes = [i32, C.POINTER(dbl)]
    L.sim_residual_screen.argtypes = [vp, i32, vp, i64, vp, vp]
    L.sim_batch_create.argtypes = [i32, C.POINTER(SimCsr), C.POINTER(SimCsr), C.POINTER(SimOptions), vp, C.POINTER(vp)]
    L.sim_batch_set_separable.argtypes = [vp, i32, i32, vp, vp]
    L.sim_batch_set_regions.argtypes = [vp, vp, vp, u64]
    L.sim_batch_solve_level.argtypes = [vp, C.POINTER(i64), C.POINTER(i32)]
    L.sim_batch_eigenvalues.argtypes = [vp, i32, vp, i64, C.POINTER(i64)]
    L.sim_batch_multiplicity.argtypes = [vp, i32, vp, i64, C.POINTER(i64)]
    L.sim_batch_handle.argtypes = [vp, i32]
    L.sim_batch_handle.restype = vp
    L.sim_batch_last_error.argtypes = [vp]
    L.sim_batch_last_error.restype = C.c_char_p
    L.sim_batch_destroy.argtypes = [vp]
    L.sim_batch_destroy.restype = None
    L.sim_solve_level.argtypes = [vp, C.POINTER(i64), C.POINTER(i32)]
    L.sim_eigenvalues.argtypes = [vp, vp, i64, C.POINTER(i64)]
    L.sim_multiplicity.argtypes = [vp, vp, i64, C.POINTER(i64)]
    L.sim_refine.argtypes = [vp, vp, vp, i64, C.POINTER(i64)]
    L.sim_projection.argtypes = [vp, i64, vp]
    L.sim_stats.argtypes = [vp, C.POINTER(SimStats), C.c_size_t]
    L.sim_last_error.argtypes = [vp]
    L.sim_last_error.restype = C.c_char_p
    L.sim_destroy.argtypes = [vp]
    L.sim_destroy.restype = None
    L.sim_shift_count.argtypes = [vp, C.POINTER(i32)]
    L.sim_get_shift.argtypes = [vp, i32, vp, vp, vp, C.POINTER(i32)]
    L.sim_eval_squares.argtypes = [vp, i32, i32, dbl, dbl, dbl, vp, vp, i64, i32, vp, vp, vp]
    L.sim_apply_shifted.argtypes = [vp, dbl, dbl, vp, vp]
    L.sim_apply_shifted_noalloc.argtypes = [vp, dbl, dbl, vp, vp]
    L.sim_shifted_solve.argtypes = [vp, dbl, dbl, vp, vp, C.POINTER(i32), C.POINTER(dbl)]
    L.sim_random_vectors.argtypes = [u64, i64, i32, i32, vp, vp]
    L.sim_kernel_timing.argtypes = [i32]
    L.sim_kernel_timing.restype = None
    L.sim_kernel_stats.argtypes = [C.c_char_p, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl), C.POINTER(i64)]
    L.sim_kernel_stats.restype = i32
    L.sim_launch_count.argtypes = []
    L.sim_launch_count.restype = i64
    for name in EXPORTS:
        f = getattr(L, name)
        if f.restype is C.c_int:  # default restype: sim_status
            f.restype = C.c_int
    _lib = L
    return L


def _check(status, handle=None):
    if status != 0:
        msg = lib().sim_last_error(handle)
        raise SimError(status, msg.decode() if msg else "")


def sim_default_options(**overrides) -> SimOptions:
    o = SimOptions()
    lib().sim_default_options(C.byref(o))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": SIM_FP64, "mixed": SIM_MIXED}[v]
        if k == "residual_scale" and isinstance(v, str):
            v = {"solution": 0, "beta": 1}[v]
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class _HostCsr:
    """Keeps host arrays alive for the duration of sim_create."""

    def __init__(self, M):
        if hasattr(M, "indptr"):
            indptr, indices, data, n = M.indptr, M.indices, M.data, M.shape[0] if hasattr(M, "shape") else M.n
        else:
            indptr, indices, data = M
            n = len(indptr) - 1
        self.indptr = np.ascontiguousarray(indptr, dtype=np.int32)
        self.indices = np.ascontiguousarray(indices, dtype=np.int32)
        self.data = np.ascontiguousarray(data, dtype=np.complex128)
        self.c = SimCsr(int(n), int(self.indices.size), self.indptr.ctypes.data, self.indices.ctypes.data,
                        self.data.ctypes.data, 0)


class _DevCsr:
    """CSR from torch tensors already on the GPU."""

    def __init__(self, indptr, indices, data):
        self.keep = (indptr, indices, data)
        self.c = SimCsr(int(indptr.numel() - 1), int(indices.numel()), indptr.data_ptr(), indices.data_ptr(),
                        data.data_ptr(), 1)


def _as_csr(M):
    if M is None:
        return None
    if isinstance(M, tuple) and len(M) == 3 and hasattr(M[0], "data_ptr") and M[0].is_cuda:
        return _DevCsr(*M)
    return _HostCsr(M)


class Sim:
    """Owns one sim_handle (see include/sim.h for the state machine)."""

    def __init__(self, A, B=None, options: SimOptions | None = None, stream=None):
        L = lib()
        self._A, self._B = _as_csr(A), _as_csr(B)
        self.options = options if options is not None else sim_default_options()
        h = C.c_void_p()
        st = L.sim_create(C.byref(self._A.c), C.byref(self._B.c) if self._B else None, C.byref(self.options),
                          _stream_ptr(stream), C.byref(h))
        _check(st, None)
        self.h = h
        self.n = self._A.c.n

    def close(self):
        if getattr(self, "h", None):
            lib().sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_separable(self, dims, axes):
        """Fast-diagonalisation preconditioner for a separable principal part:
        dims = axis lengths (axis 0 fastest), axes = [(sub, diag, sup), ...]
        complex per axis (include/sim.h, sim_set_separable)."""
        d = np.ascontiguousarray(dims, dtype=np.int64)
        a = np.ascontiguousarray(np.asarray(axes, dtype=np.complex128).reshape(-1))
        assert a.size == 3 * d.size
        _check(lib().sim_set_separable(self.h, int(d.size), d.ctypes.data, a.ctypes.data), self.h)

    def _vec_arg(self, v):
        """(pointer, on_device, keep-alive) of a complex128 vector: a CUDA
        tensor is passed as a device pointer, anything else as host memory."""
        if hasattr(v, "data_ptr") and v.is_cuda:
            return v.data_ptr(), 1, v
        a = np.ascontiguousarray(v, dtype=np.complex128)
        return a.ctypes.data, 0, a

    def projection_norm(self, center, radius, f, nodes=16, keep=True):
        """Φ = ||P f||² on the circle (center, radius) (sim_projection_norm)."""
        ptr, dev, _keep = self._vec_arg(f)
        phi = C.c_double()
        _check(lib().sim_projection_norm(self.h, float(np.real(center)), float(np.imag(center)), float(radius),
                                         int(nodes), ptr, dev, 1 if keep else 0, C.byref(phi)), self.h)
        return phi.value

    def projection_norm_grad(self, nnz_A, nnz_B=0, device=False):
        """Gradients of the last projection_norm's Φ on A's (and B's) stored
        entries, ∂Φ/∂Re + i ∂Φ/∂Im; torch CUDA tensors if device else numpy."""
        if device:
            import torch

            gA = torch.empty(nnz_A, dtype=torch.complex128, device="cuda")
            gB = torch.empty(max(nnz_B, 1), dtype=torch.complex128, device="cuda")
            _check(lib().sim_projection_norm_grad(self.h, gA.data_ptr(), gB.data_ptr() if nnz_B else None, 1), self.h)
            return gA, (gB if nnz_B else None)
        gA = np.zeros(nnz_A, dtype=np.complex128)
        gB = np.zeros(max(nnz_B, 1), dtype=np.complex128)
        _check(lib().sim_projection_norm_grad(self.h, gA.ctypes.data, gB.ctypes.data if nnz_B else None, 0), self.h)
        return gA, (gB if nnz_B else None)

    def eigenvalue_grad(self, center, radius, nnz_A, nnz_B=0, nodes=16, seed=0x5EED, device=False):
        """A simple eigenvalue inside (center, radius) and dλ/dA, dλ/dB on the
        stored entries (sim_eigenvalue_grad)."""
        lam = np.zeros(2)
        if device:
            import torch

            dA = torch.empty(nnz_A, dtype=torch.complex128, device="cuda")
            dB = torch.empty(max(nnz_B, 1), dtype=torch.complex128, device="cuda")
            pa, pb = dA.data_ptr(), (dB.data_ptr() if nnz_B else None)
        else:
            dA = np.zeros(nnz_A, dtype=np.complex128)
            dB = np.zeros(max(nnz_B, 1), dtype=np.complex128)
            pa, pb = dA.ctypes.data, (dB.ctypes.data if nnz_B else None)
        _check(lib().sim_eigenvalue_grad(self.h, float(np.real(center)), float(np.imag(center)), float(radius),
                                         int(nodes), int(seed), lam.ctypes.data, pa, pb, 1 if device else 0), self.h)
        return complex(lam[0], lam[1]), dA, (dB if nnz_B else None)

    def update_values(self, a_values=None, b_values=None):
        """New values on A's / B's stored entries (same patterns)."""
        pa = self._vec_arg(a_values) if a_values is not None else (None, 0, None)
        pb = self._vec_arg(b_values) if b_values is not None else (None, 0, None)
        dev = pa[1] if a_values is not None else pb[1]
        _check(lib().sim_update_values(self.h, pa[0], pb[0], dev), self.h)

    def set_region(self, region, f=None, seed=0):
        re_lo, re_hi, im_lo, im_hi = (float(x) for x in region)
        if f is None:
            ptr, dev = None, 0
        elif hasattr(f, "data_ptr"):
            assert f.is_cuda and f.numel() == self.n
            ptr, dev = f.data_ptr(), 1
            self._f = f
        else:
            self._f = np.ascontiguousarray(f, dtype=np.complex128)
            assert self._f.size == self.n
            ptr, dev = self._f.ctypes.data, 0
        _check(lib().sim_set_region(self.h, re_lo, re_hi, im_lo, im_hi, ptr, dev, int(seed)), self.h)

    def solve_level(self):
        nm, done = C.c_int64(), C.c_int32()
        _check(lib().sim_solve_level(self.h, C.byref(nm), C.byref(done)), self.h)
        return nm.value, bool(done.value)

    def solve_all_levels(self):
        counts = []
        while True:
            nm, done = self.solve_level()
            counts.append(nm)
            if done:
                return counts

    def eigenvalues(self) -> np.ndarray:
        cnt = C.c_int64()
        _check(lib().sim_eigenvalues(self.h, None, 0, C.byref(cnt)), self.h)
        out = np.zeros(cnt.value, dtype=np.complex128)
        if cnt.value:
            _check(lib().sim_eigenvalues(self.h, out.ctypes.data, cnt.value, C.byref(cnt)), self.h)
        return out

    def multiplicity(self) -> np.ndarray:
        cnt = C.c_int64()
        _check(lib().sim_multiplicity(self.h, None, 0, C.byref(cnt)), self.h)
        out = np.zeros(cnt.value, dtype=np.int32)
        if cnt.value:
            _check(lib().sim_multiplicity(self.h, out.ctypes.data, cnt.value, C.byref(cnt)), self.h)
        return out

    def refine(self):
        """Ritz-refined eigenvalues (same order as eigenvalues()) and a bool
        array telling which were refined."""
        cnt = C.c_int64()
        _check(lib().sim_refine(self.h, None, None, 0, C.byref(cnt)), self.h)
        out = np.zeros(cnt.value, dtype=np.complex128)
        flags = np.zeros(cnt.value, dtype=np.int32)
        if cnt.value:
            _check(lib().sim_refine(self.h, out.ctypes.data, flags.ctypes.data, cnt.value, C.byref(cnt)), self.h)
        return out, flags.astype(bool)

    def projection(self, c: int) -> np.ndarray:
        """P f onto the eigenspace of located eigenvalue c (an eigenvector
        for a simple eigenvalue), complex128[n]."""
        out = np.zeros(self.n, dtype=np.complex128)
        _check(lib().sim_projection(self.h, int(c), out.ctypes.data), self.h)
        return out

    def stats(self) -> dict:
        s = SimStats()
        _check(lib().sim_stats(self.h, C.byref(s), C.sizeof(s)), self.h)
        return s.as_dict()

    def shift_count(self) -> int:
        c = C.c_int32()
        _check(lib().sim_shift_count(self.h, C.byref(c)), self.h)
        return c.value

    def get_shift(self, s):
        m = self.options.m
        sig = np.zeros(2)
        H = np.zeros((m, m + 1), dtype=np.complex128)  # column-major (m+1) x m
        beta = np.zeros(1)
        me = C.c_int32()
        _check(lib().sim_get_shift(self.h, int(s), sig.ctypes.data, H.ctypes.data, beta.ctypes.data, C.byref(me)),
               self.h)
        return complex(sig[0], sig[1]), H.T.copy(), float(beta[0]), me.value

    def residual_screen(self, s, z):
        """e_m^T y and the β-relative residual at points z from shift s's
        eigendecomposition (Sec. 3.2, sim_residual_screen)."""
        z = np.ascontiguousarray(z, dtype=np.complex128)
        ym = np.zeros(z.size, dtype=np.complex128)
        rho = np.zeros(z.size)
        _check(lib().sim_residual_screen(self.h, int(s), z.ctypes.data, z.size, ym.ctypes.data, rho.ctypes.data),
               self.h)
        return ym, rho

    def apply_shifted(self, sigma, x):
        import torch

        y = torch.empty_like(x)
        _check(lib().sim_apply_shifted(self.h, float(np.real(sigma)), float(np.imag(sigma)), x.data_ptr(),
                                       y.data_ptr()), self.h)
        return y

    def shifted_solve(self, sigma, r):
        import torch

        x = torch.empty_like(r)
        it, rel = C.c_int32(), C.c_double()
        _check(lib().sim_shifted_solve(self.h, float(np.real(sigma)), float(np.imag(sigma)), r.data_ptr(),
                                       x.data_ptr(), C.byref(it), C.byref(rel)), self.h)
        return x, it.value, rel.value


def _bcheck(status, b):
    if status != 0:
        msg = lib().sim_batch_last_error(b)
        raise SimError(status, msg.decode() if msg else "")


class Batch:
    """Owns one sim_batch (include/sim.h): many pencils located together, every
    pencil's squares of a level evaluated in one launch."""

    def __init__(self, As, Bs=None, options: SimOptions | None = None, stream=None):
        L = lib()
        self._A = [_as_csr(a) for a in As]
        self._B = [_as_csr(b) for b in Bs] if Bs is not None else None
        arrA = (SimCsr * len(As))(*[a.c for a in self._A])
        arrB = (SimCsr * len(As))(*[b.c for b in self._B]) if self._B is not None else None
        self.options = options if options is not None else sim_default_options()
        h = C.c_void_p()
        _bcheck(L.sim_batch_create(len(As), arrA, arrB, C.byref(self.options), _stream_ptr(stream), C.byref(h)), None)
        self.h = h
        self.count = len(As)
        self.n = [a.c.n for a in self._A]

    def close(self):
        if getattr(self, "h", None):
            lib().sim_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_separable(self, p, dims, axes):
        d = np.ascontiguousarray(dims, dtype=np.int64)
        a = np.ascontiguousarray(np.asarray(axes, dtype=np.complex128).reshape(-1))
        _bcheck(lib().sim_batch_set_separable(self.h, int(p), int(d.size), d.ctypes.data, a.ctypes.data), self.h)

    def set_regions(self, regions, fs=None, seed=0):
        r = np.ascontiguousarray(np.asarray(regions, dtype=np.float64).reshape(-1))
        assert r.size == 4 * self.count
        if fs is None:
            ptr = None
        else:
            self._f = [np.ascontiguousarray(f, dtype=np.complex128) for f in fs]
            arr = (C.c_void_p * self.count)(*[f.ctypes.data for f in self._f])
            self._farr = arr
            ptr = C.cast(arr, C.c_void_p)
        _bcheck(lib().sim_batch_set_regions(self.h, r.ctypes.data, ptr, int(seed)), self.h)

    def solve_all_levels(self):
        counts = []
        while True:
            nm, done = C.c_int64(), C.c_int32()
            _bcheck(lib().sim_batch_solve_level(self.h, C.byref(nm), C.byref(done)), self.h)
            counts.append(nm.value)
            if done.value:
                return counts

    def eigenvalues(self, p) -> np.ndarray:
        cnt = C.c_int64()
        _bcheck(lib().sim_batch_eigenvalues(self.h, int(p), None, 0, C.byref(cnt)), self.h)
        out = np.zeros(cnt.value, dtype=np.complex128)
        if cnt.value:
            _bcheck(lib().sim_batch_eigenvalues(self.h, int(p), out.ctypes.data, cnt.value, C.byref(cnt)), self.h)
        return out

    def multiplicity(self, p) -> np.ndarray:
        cnt = C.c_int64()
        _bcheck(lib().sim_batch_multiplicity(self.h, int(p), None, 0, C.byref(cnt)), self.h)
        out = np.zeros(cnt.value, dtype=np.int32)
        if cnt.value:
            _bcheck(lib().sim_batch_multiplicity(self.h, int(p), out.ctypes.data, cnt.value, C.byref(cnt)), self.h)
        return out

    def stats(self, p) -> dict:
        s = SimStats()
        hp = lib().sim_batch_handle(self.h, int(p))
        _check(lib().sim_stats(hp, C.byref(s), C.sizeof(s)), hp)
        return s.as_dict()


def run(A, B, region, f, options: SimOptions | None = None, multiplicity=True, stream=None):
    """The whole SIM-M sequence; returns (eigenvalues, multiplicities or None, stats)."""
    s = Sim(A, B, options, stream)
    try:
        s.set_region(region, f)
        s.solve_all_levels()
        eig = s.eigenvalues()
        mult = s.multiplicity() if multiplicity else None
        return eig, mult, s.stats()
    finally:
        s.close()


def eval_squares(H, m_eff, beta, sigma, centers, sides, residual_scale=0, stream=None):
    """Component entry: indicator and max residual of squares against one
    Krylov space.  H: (m+1) x m complex128 numpy array; centers complex,
    sides real (numpy).  Runs on the GPU (torch provides device memory)."""
    import torch

    H = np.asarray(H, dtype=np.complex128)
    m = H.shape[1]
    dev = torch.device("cuda")
    Hd = torch.from_numpy(np.ascontiguousarray(H.T)).to(dev)  # column-major (m+1) x m
    cd = torch.from_numpy(np.ascontiguousarray(centers, dtype=np.complex128)).to(dev)
    sd = torch.from_numpy(np.ascontiguousarray(sides, dtype=np.float64)).to(dev)
    ind = torch.empty(cd.numel(), dtype=torch.float64, device=dev)
    rho = torch.empty_like(ind)
    st = lib().sim_eval_squares(Hd.data_ptr(), int(m), int(m_eff), float(beta), float(np.real(sigma)),
                                float(np.imag(sigma)), cd.data_ptr(), sd.data_ptr(), int(cd.numel()),
                                int(residual_scale), ind.data_ptr(), rho.data_ptr(), _stream_ptr(stream))
    _check(st, None)
    return ind.cpu().numpy(), rho.cpu().numpy()


def kernel_timing(enable: bool):
    lib().sim_kernel_timing(1 if enable else 0)


def kernel_stats(name: str):
    ms, by, fl, ln = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
    if not lib().sim_kernel_stats(name.encode(), C.byref(ms), C.byref(by), C.byref(fl), C.byref(ln)):
        return None
    return {"ms": ms.value, "bytes": by.value, "flops": fl.value, "launches": ln.value}


def measure_fma_peak(fp64: bool = True) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (FP64 or FP32)."""
    v = C.c_double()
    _check(lib().sim_measure_fma_peak(0 if fp64 else 1, C.byref(v)), None)
    return v.value


def launch_count() -> int:
    return int(lib().sim_launch_count())


def random_vectors(seed, n, k, first=0, stream=None):
    """Philox4x64-10 complex Gaussian vectors, shape (k, n), on the GPU."""
    import torch

    out = torch.empty((k, n), dtype=torch.complex128, device="cuda")
    _check(lib().sim_random_vectors(int(seed), int(n), int(k), int(first), out.data_ptr(), _stream_ptr(stream)),
           None)
    return out
