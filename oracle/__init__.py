"""ctypes wrapper around the FP64 CPU oracle (``ac_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The library path never imports it.

The oracle is compiled from source with gcc (``-O2 -ffp-contract=off``, no
fast-math) into ``oracle/liborc.so`` on first use, or by :func:`build`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ac_oracle.c")
_HDR = os.path.join(_HERE, "ac_oracle.h")
_LIB = os.path.join(_HERE, "liborc.so")

OK, NOT_CONVERGED, ERR_NONFINITE = 0, 1, -3
_BC = {"slip": 0, "noslip": 1, "transmissive": 2, "periodic": 3}
_RIEMANN = {"osher": 0, "bassi": 1, "roe": 2}
_GRADP = {"new": 0, "minmod": 1, "superbee": 2, "split_minmod": 3, "split_superbee": 4}


class Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double),
        ("beta", C.c_double),
        ("bc", C.c_int * 4),
        ("s_max", C.c_int), ("riemann", C.c_int), ("gradp", C.c_int), ("limiter_k", C.c_int),
        ("local_dtau", C.c_int), ("realtime", C.c_int), ("bdf_order", C.c_int),
        ("alpha_pi_p_row", C.c_int),
        ("cfl_tau", C.c_double),
        ("abs_tol", C.c_double * 4),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        for name in ("orc_flux_x", "orc_osher_x", "orc_roe_x", "orc_bassi_x"):
            fn = getattr(L, name)
            if name == "orc_flux_x":
                fn.argtypes = [_D, C.c_double, _D]
            else:
                fn.argtypes = [_D, _D, C.c_double, _D]
            fn.restype = None
        L.orc_jacobian_x.argtypes = [_D, C.c_double, _D]
        L.orc_eigen_x.argtypes = [_D, C.c_double, _D, _D, _D]
        L.orc_bassi_star.argtypes = [_D, _D, C.c_double, _D]
        L.orc_bassi_sample.argtypes = [_D, _D, C.c_double, C.c_double, _D]
        L.orc_rotation.argtypes = [_D, _D]
        L.orc_face_flux.argtypes = [_D, _D, _D, C.c_double, C.c_int, _D]
        L.orc_limiter.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_limiter.restype = C.c_double
        L.orc_bracket.argtypes = [C.POINTER(Problem), C.POINTER(_D), C.POINTER(_D), _D, C.POINTER(_D)]
        L.orc_dtau.argtypes = [C.POINTER(Problem), C.POINTER(_D), _D]
        L.orc_realtime_dt.argtypes = [C.POINTER(Problem), C.POINTER(_D), C.c_double]
        L.orc_realtime_dt.restype = C.c_double
        L.orc_physical_step.argtypes = [C.POINTER(Problem), C.POINTER(_D), C.c_void_p, C.c_double,
                                        C.c_double, C.c_int, C.POINTER(C.c_int), _D, _D]
        L.orc_physical_step.restype = C.c_int
        L.orc_pseudo_time_run.argtypes = [C.POINTER(Problem), C.POINTER(_D), C.c_double, C.c_int,
                                          C.POINTER(C.c_int)]
        L.orc_pseudo_time_run.restype = C.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _vec(x, n) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))


# ---------------------------------------------------------------- primitives

def flux_x(Q, beta):
    Q = _vec(Q, 5); F = np.zeros(5)
    lib().orc_flux_x(_p(Q), beta, _p(F)); return F


def jacobian_x(Q, beta):
    Q = _vec(Q, 5); A = np.zeros(25)
    lib().orc_jacobian_x(_p(Q), beta, _p(A)); return A.reshape(5, 5)


def eigen_x(Q, beta):
    Q = _vec(Q, 5); lam = np.zeros(5); R = np.zeros(25); L = np.zeros(25)
    lib().orc_eigen_x(_p(Q), beta, _p(lam), _p(R), _p(L))
    return lam, R.reshape(5, 5), L.reshape(5, 5)


def riemann_flux(kind: str, QL, QR, beta):
    QL = _vec(QL, 5); QR = _vec(QR, 5); F = np.zeros(5)
    getattr(lib(), f"orc_{kind}_x")(_p(QL), _p(QR), beta, _p(F)); return F


def bassi_star(WL, WR, beta):
    WL = _vec(WL, 4); WR = _vec(WR, 4); out = np.zeros(6)
    lib().orc_bassi_star(_p(WL), _p(WR), beta, _p(out)); return out


def bassi_sample(WL, WR, beta, xi):
    WL = _vec(WL, 4); WR = _vec(WR, 4); W = np.zeros(4)
    lib().orc_bassi_sample(_p(WL), _p(WR), beta, float(xi), _p(W)); return W


def rotation(n):
    n = _vec(n, 3); R = np.zeros(25)
    lib().orc_rotation(_p(n), _p(R)); return R.reshape(5, 5)


def face_flux(Qa, Qb, n, beta, riemann="osher"):
    Qa = _vec(Qa, 5); Qb = _vec(Qb, 5); n = _vec(n, 3); F = np.zeros(5)
    lib().orc_face_flux(_p(Qa), _p(Qb), _p(n), beta, _RIEMANN[riemann], _p(F)); return F


def limiter(a, b, k):
    return lib().orc_limiter(float(a), float(b), float(k))


# ------------------------------------------------------------------ problems

def problem(case, **override) -> Problem:
    """Build the oracle's problem struct from a workloads.Case."""
    o = case.options
    pb = Problem()
    pb.nx, pb.ny = case.nx, case.ny
    pb.dx, pb.dy = case.dx, case.dy
    pb.gx, pb.gy = case.gx, case.gy
    pb.beta = case.beta
    for k in range(4):
        pb.bc[k] = _BC[case.bc[k]]
    pb.s_max = o.s_max
    pb.riemann = _RIEMANN[o.riemann]
    pb.gradp = _GRADP[o.gradp]
    pb.limiter_k = o.limiter_k
    pb.local_dtau = int(o.local_dtau)
    pb.realtime = int(o.realtime)
    pb.bdf_order = o.bdf_order
    pb.alpha_pi_p_row = int(o.alpha_pi_p_row)
    pb.cfl_tau = o.cfl_tau
    for k in range(4):
        pb.abs_tol[k] = o.abs_tol[k]
    for k, v in override.items():
        setattr(pb, k, v)
    return pb


def _ptrs(arrs):
    return (_D * len(arrs))(*[_p(a) for a in arrs])


class Result(Tuple):
    pass


def physical_step(case, state, dt: Optional[float] = None, tol: Optional[float] = None,
                  max_iters: Optional[int] = None, history: Optional[Sequence] = None, **override):
    """Advance ``state`` (rho, rhou, rhov, p; each (ny, nx)) by one physical step.

    Returns (new_state, status, iterations, R, R0).  ``history`` optionally
    holds Q^{n-1} (and Q^{n-2}) as (rho, rhou, rhov) triples for BDF2/3."""
    pb = problem(case, **override)
    q = [np.ascontiguousarray(np.array(a, dtype=np.float64)) for a in state]
    its = C.c_int(0)
    R = np.zeros(4); R0 = np.zeros(4)
    hist_c = None
    keep = []
    if history:
        H = ((_D * 3) * 2)()
        for l, lev in enumerate(history[:2]):
            for f in range(3):
                a = np.ascontiguousarray(np.array(lev[f], dtype=np.float64))
                keep.append(a)
                H[l][f] = _p(a)
        hist_c = C.cast(C.pointer(H), C.c_void_p)
    st = lib().orc_physical_step(C.byref(pb), _ptrs(q), hist_c,
                                 case.dt if dt is None else dt,
                                 case.tol if tol is None else tol,
                                 case.max_iters if max_iters is None else max_iters,
                                 C.byref(its), _p(R), _p(R0))
    return tuple(q), st, its.value, R, R0


def bracket(case, state, rt=None, rho0=None, **override):
    pb = problem(case, **override)
    q = [np.ascontiguousarray(np.array(a, dtype=np.float64)) for a in state]
    br = [np.zeros_like(q[0]) for _ in range(4)]
    rtc = None
    if rt is not None:
        rt = [np.ascontiguousarray(np.array(a, dtype=np.float64)) for a in rt]
        rtc = _ptrs(rt)
    r0 = q[0] if rho0 is None else np.ascontiguousarray(np.array(rho0, dtype=np.float64))
    lib().orc_bracket(C.byref(pb), _ptrs(q), rtc, _p(r0), _ptrs(br))
    return tuple(br)


def dtau(case, state, **override):
    pb = problem(case, **override)
    q = [np.ascontiguousarray(np.array(a, dtype=np.float64)) for a in state]
    out = np.zeros_like(q[0])
    lib().orc_dtau(C.byref(pb), _ptrs(q), _p(out))
    return out


def realtime_dt(case, state, cfl_t: float, **override) -> float:
    pb = problem(case, **override)
    q = [np.ascontiguousarray(np.array(a, dtype=np.float64)) for a in state]
    return lib().orc_realtime_dt(C.byref(pb), _ptrs(q), float(cfl_t))


def pseudo_time_run(case, state, tau_end: float, max_iters: int = 1000000, **override):
    pb = problem(case, **override)
    q = [np.ascontiguousarray(np.array(a, dtype=np.float64)) for a in state]
    its = C.c_int(0)
    st = lib().orc_pseudo_time_run(C.byref(pb), _ptrs(q), float(tau_end), int(max_iters), C.byref(its))
    return tuple(q), st, its.value


def run(case, steps: Optional[int] = None, **kw):
    """Run ``steps`` physical steps from the case's initial state."""
    state = case.state()
    info = []
    for _ in range(case.steps if steps is None else steps):
        state, st, its, R, R0 = physical_step(case, state, **kw)
        info.append((st, its, R, R0))
    return state, info
