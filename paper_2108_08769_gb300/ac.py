"""Thin ctypes binding of the C ABI in ``include/ac.h`` (same names).

Argument marshalling only: every step of the sweep runs in the CUDA library
``libacgb300.so``.  There is no CPU fallback; loading fails loudly when the
library is missing or cannot be built.

``Tank`` wraps one ``ac_ctx`` for Python callers; the module-level
``ac_*`` functions mirror the C entry points one to one.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

AC_OK = 0
AC_NOT_CONVERGED = 1
AC_ERR_ARG = -1
AC_ERR_CUDA = -2
AC_ERR_NONFINITE = -3
AC_ERR_TIMEOUT = -4
AC_ERR_OOM = -5
AC_ERR_STATE = -6

BC = {"slip": 0, "noslip": 1, "transmissive": 2, "periodic": 3}
GRADP = {"new": 0, "minmod": 1, "superbee": 2, "split_minmod": 3, "split_superbee": 4}
RIEMANN = {"osher": 0, "bassi": 1, "roe": 2}
PRECISION = {"fp64": 0, "mixed": 1}

# every entry point include/ac.h declares
EXPORTS = (
    "ac_default_options", "ac_beta_from_speed", "ac_create", "ac_destroy", "ac_set_stream",
    "ac_set_state", "ac_get_state", "ac_physical_step", "ac_residual_norms", "ac_get_history",
    "ac_set_history", "ac_kernel_launches", "ac_last_error", "ac_set_profiling", "ac_stage_kernel_time",
    "ac_tile_shape", "ac_probe_fp64_fma_tflops",
    "ac_stage_sweep_noalloc", "ac_realtime_dt", "ac_pseudo_time_run", "ac_batch_create", "ac_batch_destroy", "ac_batch_set_stream",
    "ac_batch_set_state", "ac_batch_get_state", "ac_batch_physical_step", "ac_batch_residual_norms",
    "ac_batch_tile_shape", "ac_batch_set_profiling", "ac_batch_stage_kernel_time", "ac_batch_kernel_launches",
)


class ac_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double)]


class ac_fluids(C.Structure):
    _fields_ = [("rho_heavy", C.c_double), ("rho_light", C.c_double)]


class ac_bc(C.Structure):
    _fields_ = [("xlo", C.c_int), ("xhi", C.c_int), ("ylo", C.c_int), ("yhi", C.c_int)]


class ac_options(C.Structure):
    _fields_ = [("rk_stages", C.c_int), ("riemann", C.c_int), ("gradp", C.c_int), ("limiter_k", C.c_int),
                ("local_dtau", C.c_int), ("realtime", C.c_int), ("alpha_pi_p_row", C.c_int),
                ("precision", C.c_int), ("cfl_tau", C.c_double), ("abs_tol", C.c_double * 4),
                ("bdf_order", C.c_int)]


_D = C.POINTER(C.c_double)
_lib = None


class ACError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libacgb300.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    L.ac_default_options.argtypes = [C.POINTER(ac_options)]
    L.ac_beta_from_speed.argtypes = [C.c_double, C.c_double]
    L.ac_beta_from_speed.restype = C.c_double
    L.ac_create.argtypes = [C.POINTER(ac_grid), C.POINTER(ac_fluids), C.c_double, C.POINTER(ac_bc),
                            C.POINTER(ac_options), C.POINTER(C.c_void_p)]
    L.ac_destroy.argtypes = [C.c_void_p]
    L.ac_destroy.restype = None
    L.ac_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.ac_set_state.argtypes = [C.c_void_p, _D, _D, _D, _D]
    L.ac_get_state.argtypes = [C.c_void_p, _D, _D, _D, _D]
    L.ac_physical_step.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.ac_pseudo_time_run.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int)]
    L.ac_residual_norms.argtypes = [C.c_void_p, _D, _D]
    L.ac_realtime_dt.argtypes = [C.c_void_p, C.c_double, _D]
    L.ac_get_history.argtypes = [C.c_void_p, C.c_int, _D, _D, _D]
    L.ac_set_history.argtypes = [C.c_void_p, C.c_int, _D, _D, _D]
    L.ac_kernel_launches.argtypes = [C.c_void_p]
    L.ac_kernel_launches.restype = C.c_longlong
    L.ac_set_profiling.argtypes = [C.c_void_p, C.c_int]
    L.ac_stage_kernel_time.argtypes = [C.c_void_p, _D, C.POINTER(C.c_longlong)]
    _IP = C.POINTER(C.c_int)
    L.ac_tile_shape.argtypes = [C.c_void_p, _IP, _IP, _IP, _IP]
    L.ac_probe_fp64_fma_tflops.argtypes = [_D]
    _PA4 = C.c_void_p * 4
    _PA3 = C.c_void_p * 3
    L.ac_stage_sweep_noalloc.argtypes = [C.POINTER(ac_grid), C.c_double, C.POINTER(ac_bc), C.POINTER(ac_options),
                                         C.c_int, C.c_double, _PA4, _PA4, _PA3, _PA4, C.c_void_p, C.c_void_p]
    _I = C.POINTER(C.c_int)
    L.ac_batch_create.argtypes = [C.c_int, C.POINTER(ac_grid), _D, C.POINTER(ac_bc), C.POINTER(ac_options),
                                  C.POINTER(C.c_void_p)]
    L.ac_batch_destroy.argtypes = [C.c_void_p]
    L.ac_batch_destroy.restype = None
    L.ac_batch_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.ac_batch_set_state.argtypes = [C.c_void_p, C.c_int, _D, _D, _D, _D]
    L.ac_batch_get_state.argtypes = [C.c_void_p, C.c_int, _D, _D, _D, _D]
    L.ac_batch_physical_step.argtypes = [C.c_void_p, _D, C.c_double, C.c_int, _I, _I]
    L.ac_batch_residual_norms.argtypes = [C.c_void_p, C.c_int, _D, _D]
    L.ac_batch_tile_shape.argtypes = [C.c_void_p, _I, _I, _I]
    L.ac_batch_set_profiling.argtypes = [C.c_void_p, C.c_int]
    L.ac_batch_stage_kernel_time.argtypes = [C.c_void_p, _D, C.POINTER(C.c_longlong)]
    L.ac_batch_kernel_launches.argtypes = [C.c_void_p]
    L.ac_batch_kernel_launches.restype = C.c_longlong
    L.ac_last_error.argtypes = []
    L.ac_last_error.restype = C.c_char_p
    _lib = L
    return L


def ac_last_error() -> str:
    return load().ac_last_error().decode()


def _check(rc: int, allow=(AC_OK,)) -> int:
    if rc not in allow:
        raise ACError(rc, ac_last_error())
    return rc


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _host(a, n) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def ac_default_options() -> ac_options:
    o = ac_options()
    _check(load().ac_default_options(C.byref(o)))
    return o


def ac_probe_fp64_fma_tflops() -> float:
    """The device's FP64 FMA rate (TFLOP/s), measured by the library."""
    v = C.c_double(0.0)
    _check(load().ac_probe_fp64_fma_tflops(C.byref(v)))
    return v.value


def ac_beta_from_speed(c0: float, rho_ref: float) -> float:
    return load().ac_beta_from_speed(c0, rho_ref)


def options_from(case_options, precision: str = "fp64") -> ac_options:
    """ac_options from a workloads.Options."""
    o = ac_default_options()
    o.rk_stages = case_options.s_max
    o.riemann = RIEMANN[case_options.riemann]
    o.gradp = GRADP[case_options.gradp]
    o.limiter_k = case_options.limiter_k
    o.local_dtau = int(case_options.local_dtau)
    o.realtime = int(case_options.realtime)
    o.alpha_pi_p_row = int(case_options.alpha_pi_p_row)
    o.precision = PRECISION[precision]
    o.cfl_tau = case_options.cfl_tau
    for k in range(4):
        o.abs_tol[k] = case_options.abs_tol[k]
    o.bdf_order = case_options.bdf_order
    return o


def ac_stage_sweep_noalloc(nx, ny, lx, ly, gx, gy, beta, bc, options, stage, dt, q_prev, q0, qn, q_out,
                           norms=0, stream=0):
    """One FP64 stage sweep on caller-owned device arrays, allocating
    nothing (see include/ac.h).  Field arguments are sequences of device
    addresses (ints); norms is a device address of 4 doubles or 0."""
    L = load()
    g = ac_grid(nx, ny, lx, ly, gx, gy)
    b = ac_bc(*[BC[s] for s in bc])
    A4 = C.c_void_p * 4
    A3 = C.c_void_p * 3
    qp = A4(*(q_prev if q_prev is not None else [0, 0, 0, 0]))
    rc = L.ac_stage_sweep_noalloc(C.byref(g), beta, C.byref(b), C.byref(options), stage, dt, qp, A4(*q0),
                                  A3(*qn) if qn is not None else None, A4(*q_out), C.c_void_p(norms or 0),
                                  C.c_void_p(stream or 0))
    _check(rc)


class Tank:
    """One simulated tank: an ``ac_ctx`` with its state on the GPU."""

    def __init__(self, nx: int, ny: int, lx: float, ly: float, gx: float, gy: float, beta: float,
                 bc: Sequence[str], options: Optional[ac_options] = None,
                 fluids: Optional[Tuple[float, float]] = None):
        L = load()
        self.nx, self.ny = nx, ny
        g = ac_grid(nx, ny, lx, ly, gx, gy)
        b = ac_bc(*[BC[s] for s in bc])
        fl = ac_fluids(fluids[0], fluids[1]) if fluids else None
        h = C.c_void_p()
        _check(L.ac_create(C.byref(g), C.byref(fl) if fl else None, beta, C.byref(b),
                           C.byref(options) if options is not None else None, C.byref(h)))
        self._h = h

    @classmethod
    def from_case(cls, case, precision: str = "fp64", fluids=None) -> "Tank":
        t = cls(case.nx, case.ny, case.lx, case.ly, case.gx, case.gy, case.beta, case.bc,
                options_from(case.options, precision), fluids)
        t.set_state(*case.state())
        return t

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ac_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr: int):
        _check(load().ac_set_stream(self._h, C.c_void_p(stream_ptr)))

    def set_state(self, rho, rhou, rhov, p):
        n = self.nx * self.ny
        arrs = [_host(a, n) for a in (rho, rhou, rhov, p)]
        _check(load().ac_set_state(self._h, *[_ptr(a) for a in arrs]))

    def get_state(self) -> Tuple[np.ndarray, ...]:
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        _check(load().ac_get_state(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def get_state_into(self, rho, rhou, rhov, p):
        """Copy the state into caller-provided (e.g. pinned) float64 arrays."""
        _check(load().ac_get_state(self._h, _ptr(rho), _ptr(rhou), _ptr(rhov), _ptr(p)))

    def physical_step(self, dt: float, tol: float, max_iters: int) -> Tuple[int, int]:
        its = C.c_int(0)
        rc = load().ac_physical_step(self._h, dt, tol, max_iters, C.byref(its))
        _check(rc, (AC_OK, AC_NOT_CONVERGED))
        return rc, its.value

    def pseudo_time_run(self, tau_end: float, max_iters: int = 1000000) -> Tuple[int, int]:
        its = C.c_int(0)
        rc = load().ac_pseudo_time_run(self._h, tau_end, max_iters, C.byref(its))
        _check(rc, (AC_OK, AC_NOT_CONVERGED))
        return rc, its.value

    def residual_norms(self) -> Tuple[np.ndarray, np.ndarray]:
        R = np.zeros(4)
        R0 = np.zeros(4)
        _check(load().ac_residual_norms(self._h, _ptr(R), _ptr(R0)))
        return R, R0

    def realtime_dt(self, cfl_t: float) -> float:
        out = C.c_double(0.0)
        _check(load().ac_realtime_dt(self._h, cfl_t, C.byref(out)))
        return out.value

    def get_history(self, k: int) -> Tuple[np.ndarray, ...]:
        out = [np.empty((self.ny, self.nx)) for _ in range(3)]
        _check(load().ac_get_history(self._h, k, *[_ptr(a) for a in out]))
        return tuple(out)

    def set_history(self, k: int, rho, rhou, rhov):
        n = self.nx * self.ny
        arrs = [_host(a, n) for a in (rho, rhou, rhov)]
        _check(load().ac_set_history(self._h, k, *[_ptr(a) for a in arrs]))

    def kernel_launches(self) -> int:
        return load().ac_kernel_launches(self._h)

    def set_profiling(self, on: bool):
        _check(load().ac_set_profiling(self._h, int(on)))

    def stage_kernel_time(self) -> Tuple[float, int]:
        ms = C.c_double(0.0)
        n = C.c_longlong(0)
        _check(load().ac_stage_kernel_time(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def tile_shape(self):
        """(tx, ty, threads, variant) of the tuned stage sweep (variant -1 before the first step)."""
        a, b, c, v = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        load().ac_tile_shape(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(v))
        return a.value, b.value, c.value, v.value


class Batch:
    """Many tanks advanced together in the mixed form (an ``ac_batch``)."""

    def __init__(self, cases, options: Optional[ac_options] = None):
        L = load()
        n = len(cases)
        self.cases = list(cases)
        grids = (ac_grid * n)(*[ac_grid(c.nx, c.ny, c.lx, c.ly, c.gx, c.gy) for c in cases])
        bcs = (ac_bc * n)(*[ac_bc(*[BC[s] for s in c.bc]) for c in cases])
        betas = (C.c_double * n)(*[c.beta for c in cases])
        if options is None:
            options = options_from(cases[0].options, "mixed")
        h = C.c_void_p()
        _check(L.ac_batch_create(n, grids, betas, bcs, C.byref(options), C.byref(h)))
        self._h = h
        self.n = n

    @classmethod
    def from_cases(cls, cases, options: Optional[ac_options] = None) -> "Batch":
        b = cls(cases, options)
        for k, c in enumerate(cases):
            b.set_state(k, *c.state())
        return b

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ac_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr: int):
        _check(load().ac_batch_set_stream(self._h, C.c_void_p(stream_ptr)))

    def set_state(self, k, rho, rhou, rhov, p):
        c = self.cases[k]
        n = c.nx * c.ny
        arrs = [_host(a, n) for a in (rho, rhou, rhov, p)]
        _check(load().ac_batch_set_state(self._h, k, *[_ptr(a) for a in arrs]))

    def get_state(self, k):
        c = self.cases[k]
        out = [np.empty((c.ny, c.nx)) for _ in range(4)]
        _check(load().ac_batch_get_state(self._h, k, *[_ptr(a) for a in out]))
        return tuple(out)

    def physical_step(self, dt, tol: float, max_iters: int):
        dts = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.n,)))
        its = (C.c_int * self.n)()
        st = (C.c_int * self.n)()
        rc = load().ac_batch_physical_step(self._h, _ptr(dts), tol, max_iters, its, st)
        _check(rc, (AC_OK, AC_NOT_CONVERGED))
        return rc, list(its), list(st)

    def residual_norms(self, k):
        R = np.zeros(4)
        R0 = np.zeros(4)
        _check(load().ac_batch_residual_norms(self._h, k, _ptr(R), _ptr(R0)))
        return R, R0

    def tile_shape(self):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        load().ac_batch_tile_shape(self._h, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def set_profiling(self, on: bool):
        _check(load().ac_batch_set_profiling(self._h, int(on)))

    def stage_kernel_time(self):
        ms = C.c_double(0.0)
        n = C.c_longlong(0)
        _check(load().ac_batch_stage_kernel_time(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def kernel_launches(self) -> int:
        return load().ac_batch_kernel_launches(self._h)
