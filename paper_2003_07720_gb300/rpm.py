"""ctypes binding of the C ABI in include/rpm.h (argument marshalling only).

The functions keep the C names.  Field arguments are torch CUDA float32
tensors of shape (6, nz, ny, nx) (contiguous) or raw device pointers; every
step of the computation runs in the CUDA library.  If the library has not
been built, loading fails loudly: there is no other implementation behind
these names.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librpmfft.so")

RPM_OK = 0
RPM_ERR_INVALID_ARG = 1
RPM_ERR_UNSUPPORTED_GRID = 2
RPM_ERR_OOM = 3
RPM_ERR_CUDA = 4
RPM_ERR_NOT_CONVERGED = 5
RPM_ERR_DIVERGED = 6
RPM_ERR_TIMEOUT = 7

RPM_NYQ_ZERO_MIXED = 0

RPM_SCHEME_BASIC = 0
RPM_SCHEME_POLARIZATION = 1

RPM_GAMMA_FULL_MAP = 0
RPM_GAMMA_LINEAR = 1
RPM_GAMMA_RAW_TAU = 2
RPM_GAMMA_PROJECT = 3


class rpm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


class rpm_iso(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("mu", ctypes.c_double)]


class rpm_options(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int), ("p_max", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("tol", ctypes.c_double), ("t_ratio", ctypes.c_double),
                ("nyquist", ctypes.c_int), ("diverge_factor", ctypes.c_double),
                ("max_device_gb", ctypes.c_double), ("profile", ctypes.c_int),
                ("scheme", ctypes.c_int), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("warm_tol", ctypes.c_double), ("warm_c0_scale", ctypes.c_double),
                ("warm_max_iters", ctypes.c_int), ("warm_p_max", ctypes.c_int),
                ("warm_from_eps0", ctypes.c_int), ("autotune", ctypes.c_int),
                ("plane_variant", ctypes.c_int), ("pencil_variant", ctypes.c_int),
                ("share_basis", ctypes.c_int)]


class rpm_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("gamma_applies", ctypes.c_int),
                ("basis_size", ctypes.c_int), ("converged", ctypes.c_int),
                ("status", ctypes.c_int), ("residual", ctypes.c_double),
                ("residual0", ctypes.c_double), ("mean_stress", ctypes.c_double * 6),
                ("ms", ctypes.c_float), ("gamma_ms", ctypes.c_float),
                ("proj_ms", ctypes.c_float), ("launches", ctypes.c_longlong),
                ("proj_bytes", ctypes.c_double), ("warm_iters", ctypes.c_int),
                ("warm_residual", ctypes.c_double), ("basis_reused", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"iters": self.iters, "gamma_applies": self.gamma_applies,
                "basis_size": self.basis_size, "converged": bool(self.converged),
                "status": self.status, "residual": self.residual,
                "residual0": self.residual0, "mean_stress": list(self.mean_stress),
                "ms": self.ms, "gamma_ms": self.gamma_ms, "proj_ms": self.proj_ms,
                "launches": self.launches, "proj_bytes": self.proj_bytes,
                "warm_iters": self.warm_iters, "warm_residual": self.warm_residual,
                "basis_reused": self.basis_reused}


class rpm_cell(ctypes.Structure):
    _fields_ = [("grid", rpm_grid), ("phase", ctypes.c_void_p), ("n_phases", ctypes.c_int),
                ("phases", ctypes.c_void_p), ("c0", rpm_iso)]


_lib = None

EXPORTS = ("rpm_default_options", "rpm_create", "rpm_set_phase", "rpm_set_options",
           "rpm_apply_gamma", "rpm_solve", "rpm_effective_stiffness", "rpm_last_error",
           "rpm_status_string", "rpm_device_bytes", "rpm_grid_supported", "rpm_destroy",
           "rpm_set_trace", "rpm_set_materials", "rpm_effective_stiffness_batch",
           "rpm_pencil_tile", "rpm_plane_variant", "rpm_bounded_wait_check")


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"RPM-FFT CUDA library not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    L.rpm_default_options.argtypes = [P(rpm_options)]
    L.rpm_default_options.restype = None
    L.rpm_create.argtypes = [P(rpm_grid), vp, ctypes.c_int, ctypes.c_int, P(rpm_iso), rpm_iso,
                             P(rpm_options), vp, P(vp)]
    L.rpm_create.restype = ctypes.c_int
    L.rpm_set_phase.argtypes = [vp, vp, ctypes.c_int]
    L.rpm_set_phase.restype = ctypes.c_int
    L.rpm_set_options.argtypes = [vp, P(rpm_options)]
    L.rpm_set_options.restype = ctypes.c_int
    L.rpm_apply_gamma.argtypes = [vp, vp, P(ctypes.c_double), vp, ctypes.c_int]
    L.rpm_apply_gamma.restype = ctypes.c_int
    L.rpm_solve.argtypes = [vp, P(ctypes.c_double), vp, vp, vp, ctypes.c_int, P(rpm_solve_info)]
    L.rpm_solve.restype = ctypes.c_int
    L.rpm_effective_stiffness.argtypes = [vp, P(ctypes.c_double), P(rpm_solve_info)]
    L.rpm_effective_stiffness.restype = ctypes.c_int
    L.rpm_last_error.argtypes = [vp]
    L.rpm_last_error.restype = ctypes.c_char_p
    L.rpm_status_string.argtypes = [ctypes.c_int]
    L.rpm_status_string.restype = ctypes.c_char_p
    L.rpm_device_bytes.argtypes = [vp]
    L.rpm_device_bytes.restype = ctypes.c_size_t
    L.rpm_grid_supported.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.rpm_grid_supported.restype = ctypes.c_int
    L.rpm_set_trace.argtypes = [vp, vp, vp, ctypes.c_int]
    L.rpm_set_trace.restype = ctypes.c_int
    L.rpm_set_materials.argtypes = [vp, ctypes.c_int, P(rpm_iso), rpm_iso]
    L.rpm_set_materials.restype = ctypes.c_int
    L.rpm_effective_stiffness_batch.argtypes = [P(rpm_cell), ctypes.c_int, P(rpm_options),
                                                ctypes.c_int, P(ctypes.c_double),
                                                P(rpm_solve_info), P(ctypes.c_int)]
    L.rpm_effective_stiffness_batch.restype = ctypes.c_int
    L.rpm_pencil_tile.argtypes = [vp]
    L.rpm_pencil_tile.restype = ctypes.c_int
    L.rpm_plane_variant.argtypes = [vp]
    L.rpm_plane_variant.restype = ctypes.c_int
    L.rpm_bounded_wait_check.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_float)]
    L.rpm_bounded_wait_check.restype = ctypes.c_int
    L.rpm_destroy.argtypes = [vp]
    L.rpm_destroy.restype = None
    _lib = L
    return L


class RpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{lib().rpm_status_string(status).decode()}: {msg}")
        self.status = status


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _E(E) -> ctypes.Array:
    a = (ctypes.c_double * 6)(*[float(v) for v in np.asarray(E, float).ravel()])
    return a


def rpm_default_options(**overrides) -> rpm_options:
    o = rpm_options()
    lib().rpm_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def rpm_grid_supported(nx: int, ny: int, nz: int) -> bool:
    return bool(lib().rpm_grid_supported(nx, ny, nz))


def rpm_create(shape, phase, phases, c0, options: rpm_options | None = None, stream=None,
               lengths=(1.0, 1.0, 1.0)) -> int:
    """shape = (nz, ny, nx); phase: uint8 torch CUDA tensor or numpy array;
    phases: sequence of (lambda, mu); c0: (lambda0, mu0).  Returns a handle."""
    nz, ny, nx = shape
    g = rpm_grid(nx, ny, nz, float(lengths[2]), float(lengths[1]), float(lengths[0]))
    arr = (rpm_iso * len(phases))(*[rpm_iso(float(l), float(m)) for (l, m) in phases])
    on_dev = int(hasattr(phase, "is_cuda") and phase.is_cuda)
    if not on_dev:
        phase = np.ascontiguousarray(np.asarray(phase, dtype=np.uint8))
    h = ctypes.c_void_p()
    st = lib().rpm_create(ctypes.byref(g), _ptr(phase), on_dev, len(phases), arr,
                          rpm_iso(float(c0[0]), float(c0[1])),
                          ctypes.byref(options) if options is not None else None,
                          _stream_ptr(stream), ctypes.byref(h))
    if st != RPM_OK:
        raise RpmError(st, "rpm_create failed")
    return h.value


def _check(ctx, st, allow=()):
    if st != RPM_OK and st not in allow:
        raise RpmError(st, lib().rpm_last_error(ctx).decode())
    return st


def rpm_set_phase(ctx, phase) -> None:
    on_dev = int(hasattr(phase, "is_cuda") and phase.is_cuda)
    if not on_dev:
        phase = np.ascontiguousarray(np.asarray(phase, dtype=np.uint8))
    _check(ctx, lib().rpm_set_phase(ctx, _ptr(phase), on_dev))


def rpm_set_options(ctx, options: rpm_options) -> None:
    _check(ctx, lib().rpm_set_options(ctx, ctypes.byref(options)))


def rpm_apply_gamma(ctx, eps_in, E, out, flags: int = RPM_GAMMA_FULL_MAP) -> None:
    _check(ctx, lib().rpm_apply_gamma(ctx, _ptr(eps_in), _E(E if E is not None else np.zeros(6)),
                                      _ptr(out), flags))


def rpm_solve(ctx, E, eps0=None, eps_out=None, sig_out=None, out_on_host: bool = False,
              raise_on_failure: bool = True) -> tuple[int, dict]:
    info = rpm_solve_info()
    st = lib().rpm_solve(ctx, _E(E), _ptr(eps0), _ptr(eps_out), _ptr(sig_out),
                         int(out_on_host), ctypes.byref(info))
    if raise_on_failure:
        _check(ctx, st)
    elif st in (RPM_ERR_INVALID_ARG, RPM_ERR_CUDA):
        _check(ctx, st)
    return st, info.as_dict()


def rpm_effective_stiffness(ctx, raise_on_failure: bool = True):
    C = (ctypes.c_double * 36)()
    infos = (rpm_solve_info * 6)()
    st = lib().rpm_effective_stiffness(ctx, C, infos)
    if raise_on_failure:
        _check(ctx, st)
    return np.array(C[:]).reshape(6, 6), [i.as_dict() for i in infos], st


def rpm_set_trace(ctx, residuals, basis_sizes, capacity: int) -> None:
    """residuals: float64 numpy array, basis_sizes: int32 numpy array (host,
    kept alive by the caller)."""
    _check(ctx, lib().rpm_set_trace(ctx, _ptr(residuals), _ptr(basis_sizes), int(capacity)))


def rpm_set_materials(ctx, phases, c0) -> None:
    arr = (rpm_iso * len(phases))(*[rpm_iso(float(l), float(m)) for (l, m) in phases])
    _check(ctx, lib().rpm_set_materials(ctx, len(phases), arr, rpm_iso(float(c0[0]), float(c0[1]))))


def rpm_effective_stiffness_batch(cells, options: rpm_options | None = None, n_workers: int = 4,
                                  raise_on_failure: bool = True):
    """cells: objects with .phase (uint8 [nz, ny, nx]), .lam, .mu, .lam0, .mu0.
    Returns (C_eff [n, 6, 6], infos [n][6] dicts, per-cell status, status)."""
    n = len(cells)
    keep = []
    arr = (rpm_cell * max(n, 1))()
    for i, c in enumerate(cells):
        ph = np.ascontiguousarray(np.asarray(c.phase, dtype=np.uint8))
        mats = (rpm_iso * len(c.lam))(*[rpm_iso(float(l), float(m)) for l, m in zip(c.lam, c.mu)])
        keep += [ph, mats]
        nz, ny, nx = ph.shape
        arr[i] = rpm_cell(rpm_grid(nx, ny, nz, 1.0, 1.0, 1.0), ph.ctypes.data, len(c.lam),
                          ctypes.cast(mats, ctypes.c_void_p).value,
                          rpm_iso(float(c.lam0), float(c.mu0)))
    C = (ctypes.c_double * (36 * max(n, 1)))()
    infos = (rpm_solve_info * (6 * max(n, 1)))()
    stat = (ctypes.c_int * max(n, 1))()
    st = lib().rpm_effective_stiffness_batch(arr, n, ctypes.byref(options) if options else None,
                                             int(n_workers), C, infos, stat)
    if raise_on_failure and st != RPM_OK:
        raise RpmError(st, "rpm_effective_stiffness_batch failed")
    return (np.array(C[:36 * n]).reshape(n, 6, 6), [[infos[6 * i + j].as_dict() for j in range(6)]
                                                   for i in range(n)], list(stat[:n]), st)


def rpm_pencil_tile(ctx) -> int:
    """Pencils per block of the z pass in use (the autotuner's choice)."""
    return int(lib().rpm_pencil_tile(ctx))


def rpm_plane_variant(ctx) -> int:
    """Plane-pass kernels in use: 0 fused, 1 whole-plane, 2 five-pass."""
    return int(lib().rpm_plane_variant(ctx))


def rpm_bounded_wait_check(stream=None) -> tuple[bool, float]:
    """Run the bounded-wait self-check on `stream`: (gave up by itself, ms waited)."""
    g, ms = ctypes.c_int(0), ctypes.c_float(0.0)
    st = lib().rpm_bounded_wait_check(_stream_ptr(stream), ctypes.byref(g), ctypes.byref(ms))
    if st != RPM_OK:
        raise RpmError(st, "bounded-wait self-check failed")
    return bool(g.value), float(ms.value)


def rpm_device_bytes(ctx) -> int:
    return int(lib().rpm_device_bytes(ctx))


def rpm_destroy(ctx) -> None:
    if ctx:
        lib().rpm_destroy(ctx)


def status_name(status: int) -> str:
    """Name of a status code (rpm_status_string)."""
    return lib().rpm_status_string(int(status)).decode()


class Context:
    """Owning wrapper around a context handle (closes on `close()` / exit)."""

    def __init__(self, cell, options: rpm_options | None = None, stream=None,
                 lengths=(1.0, 1.0, 1.0), phase=None):
        phases = list(zip(np.asarray(cell.lam, float), np.asarray(cell.mu, float)))
        self.shape = tuple(cell.phase.shape)
        self.handle = rpm_create(self.shape, cell.phase if phase is None else phase, phases,
                                 (cell.lam0, cell.mu0), options, stream, lengths)

    def apply_gamma(self, eps_in, E, out, flags=RPM_GAMMA_FULL_MAP):
        rpm_apply_gamma(self.handle, eps_in, E, out, flags)

    def solve(self, E, **kw):
        return rpm_solve(self.handle, E, **kw)

    def effective_stiffness(self, **kw):
        return rpm_effective_stiffness(self.handle, **kw)

    def trace(self, capacity: int = 10000):
        """Start recording residual / basis-size histories; returns the arrays."""
        self._trace = (np.full(capacity, np.nan), np.full(capacity, -1, dtype=np.int32))
        rpm_set_trace(self.handle, self._trace[0], self._trace[1], capacity)
        return self._trace

    def close(self):
        if self.handle:
            rpm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
