"""Parity at the largest workload size on sampled outputs.

The Rayleigh-Taylor tank (2048 x 8192 cells) is too large for the oracle as
a whole, but after one pseudo-iteration an output cell depends only on the
input within 6 cells of it (3 stages of a two-cell stencil; the real-time
term and the pseudo-time step are cell-local or one-cell wide).  So the
oracle, run on a window of the grid whose sides lying on the domain edge
keep the domain's boundary kind (the other sides are transmissive), gives
the exact full-grid result on the window's cells more than 8 cells from an
artificial side.  Several windows (interior, corners, walls, the interface)
are compared with the GPU run on the full grid in the benchmark's launch
configuration.
"""
import numpy as np
import pytest

import oracle
from conftest import rel_errors
from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MARGIN = 8


def window(case, i0, j0, w, h):
    bc = (case.bc[0] if i0 == 0 else "transmissive",
          case.bc[1] if i0 + w == case.nx else "transmissive",
          case.bc[2] if j0 == 0 else "transmissive",
          case.bc[3] if j0 + h == case.ny else "transmissive")
    sl = (slice(j0, j0 + h), slice(i0, i0 + w))
    sub = W.Case(f"win_{i0}_{j0}", w, h, w * case.dx, h * case.dy, case.gx, case.gy, case.beta, bc,
                 case.rho[sl].copy(), case.rhou[sl].copy(), case.rhov[sl].copy(), case.p[sl].copy(),
                 dt=case.dt, options=case.options)
    # compared region: away from the artificial sides
    ci = slice(0 if i0 == 0 else MARGIN, w if i0 + w == case.nx else w - MARGIN)
    cj = slice(0 if j0 == 0 else MARGIN, h if j0 + h == case.ny else h - MARGIN)
    return sub, sl, (cj, ci)


@pytest.fixture(scope="module")
def rt_case():
    return W.rayleigh_taylor(2048, 8192)


def windows_of(case):
    w = h = 48
    nx, ny = case.nx, case.ny
    return [(0, 0), (nx - w, ny - h), (0, ny // 2 - h // 2), (nx // 2, ny // 2 - h // 2),
            (777, 4080), (1500, 123), (nx - w, 4000)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
def test_rayleigh_taylor_full_grid_sampled_windows(rt_case, precision, tol):
    case = rt_case
    t = ac.Tank.from_case(case, precision=precision)
    t.physical_step(case.dt, -1.0, 1)
    full = t.get_state()
    t.close()
    for i0, j0 in windows_of(case):
        sub, sl, (cj, ci) = window(case, i0, j0, 48, 48)
        ref, *_ = oracle.physical_step(sub, sub.state(), tol=-1.0, max_iters=1)
        got = tuple(f[sl][cj, ci] for f in full)
        exp = tuple(r[cj, ci] for r in ref)
        errs = rel_errors(got, exp)
        assert max(errs) <= tol, ((i0, j0), errs)


def test_batched_64_tanks_full_size():
    """The batched benchmark's 64 tanks (64^2..1024^2, mixed form) in the
    launch configuration the benchmark times, one physical step of one
    pseudo-iteration: the three smallest tanks whole against the oracle, and
    windows of the three largest (same dependency margin as above)."""
    cases = W.batched_tanks(count=64, nmin=64, nmax=1024)
    b = ac.Batch.from_cases(cases)
    rc, its, st = b.physical_step([c.dt for c in cases], -1.0, 1)
    assert its == [1] * len(cases)
    order = sorted(range(len(cases)), key=lambda k: cases[k].cells)
    for k in order[:3]:
        c = cases[k]
        ref, *_ = oracle.physical_step(c, c.state(), tol=-1.0, max_iters=1)
        errs = rel_errors(b.get_state(k), ref)
        assert max(errs) <= 1e-5, (k, c.nx, errs)
    for k in order[-3:]:
        c = cases[k]
        full = b.get_state(k)
        for i0, j0 in [(0, 0), (c.nx - 48, c.ny - 48), (c.nx // 2, c.ny // 3)]:
            sub, sl, (cj, ci) = window(c, i0, j0, 48, 48)
            ref, *_ = oracle.physical_step(sub, sub.state(), tol=-1.0, max_iters=1)
            got = tuple(f[sl][cj, ci] for f in full)
            errs = rel_errors(got, tuple(r[cj, ci] for r in ref))
            assert max(errs) <= 1e-5, (k, (i0, j0), errs)
    b.close()
