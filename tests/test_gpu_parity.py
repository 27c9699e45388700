"""GPU FP64 sweep vs the FP64 oracle, element by element, through the C ABI.

Bar: relative L-infinity error <= 1e-11 per field after one physical step
from an identical input state (every field, each momentum component
separately, against its own largest magnitude; momentum scales at least
max(rho) * 1e-3 m/s), and identical pseudo-iteration counts when the
stopping test ends the step.  Sizes span several 32x8 tiles with ragged tails; options cover
every boundary kind, pressure-gradient method, limiter, stage count and
pseudo-time-step mode.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import rel_errors
from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-11


def run_both(case, steps=1, tol=None, max_iters=None):
    """Advance GPU and oracle from the same state, one physical step at a
    time; each step starts both from the oracle's previous state."""
    t = ac.Tank.from_case(case)
    state = case.state()
    out = []
    for _ in range(steps):
        t.set_state(*state)
        rc, its = t.physical_step(case.dt, case.tol if tol is None else tol,
                                  case.max_iters if max_iters is None else max_iters)
        got = t.get_state()
        R, R0 = t.residual_norms()
        ref, st, oits, oR, oR0 = oracle.physical_step(case, state, tol=tol, max_iters=max_iters)
        out.append((got, ref, rc, its, st, oits, R, oR, R0, oR0))
        state = ref
    t.close()
    return out


def norm_atol(ref, case):
    """Absolute floor for comparing residual norms: 1e-12 of the size of the
    individual terms that cancel in the bracket (flux differences over a
    cell), so norms at round-off level are compared against that level."""
    rho, p = ref[0], ref[3]
    h = min(case.dx, case.dy)
    b = case.beta
    mom = (np.abs(p).max() + 4.0 * b) / h
    return 1e-12 * np.array([math.sqrt(4.0 * b * rho.max()) / h, mom, mom,
                             b * math.sqrt(4.0 * b / rho.min()) / h])


def assert_parity(res, tol=TOL, check_iters=True, case=None):
    for got, ref, rc, its, st, oits, R, oR, R0, oR0 in res:
        errs = rel_errors(got, ref)
        assert max(errs) <= tol, errs
        if check_iters:
            assert its == oits, (its, oits)
            assert rc == st, (rc, st)
        atol = norm_atol(ref, case) if case is not None else 0.0
        assert np.all(np.abs(R - oR) <= 1e-9 * np.abs(oR) + atol), (R, oR, atol)
        assert np.all(np.abs(R0 - oR0) <= 1e-9 * np.abs(oR0) + atol), (R0, oR0, atol)


def test_riemann_200x4_converged_steps():
    """1D density-discontinuity Riemann problem (200x4, periodic in y,
    transmissive in x): two physical steps ending on the 1e-8 residual drop."""
    case = W.riemann_tank()
    assert_parity(run_both(case, steps=2), case=case)


def test_hydrostatic_tank_64_fixed_iterations():
    case = W.hydrostatic_tank(64)
    res = run_both(case, steps=1, tol=-1.0, max_iters=12)
    assert_parity(res, case=case)
    got = res[0][0]
    assert np.abs(got[2]).max() < 1e-10


def test_hydrostatic_tank_256_full_size():
    """The benchmarked 256x256 workload in the benchmark's launch
    configuration, a few pseudo-iterations, against the oracle on every cell."""
    case = W.hydrostatic_tank(256)
    assert_parity(run_both(case, steps=1, tol=-1.0, max_iters=3), case=case)


def test_water_column_1024x512_full_size_one_iteration():
    case = W.water_column(1024, 512)
    assert_parity(run_both(case, steps=1, tol=-1.0, max_iters=1), case=case)


BCS = [("slip",) * 4,
       ("noslip",) * 4,
       ("transmissive", "slip", "noslip", "transmissive"),
       ("periodic", "periodic", "slip", "slip"),
       ("slip", "noslip", "periodic", "periodic"),
       ("periodic",) * 4]


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("nx,ny", [(37, 19), (70, 9), (5, 3)])
def test_boundary_kinds_ragged_grids(bc, nx, ny):
    case = W.random_two_fluid(nx, ny, ratio=500.0, c0=8.0, bc=bc, gx=1.5,
                              gy=0.0 if bc[2] == "periodic" else -9.81)
    assert_parity(run_both(case, steps=1, tol=-1.0, max_iters=4), case=case)


OPTION_SETS = [
    dict(gradp="minmod"),
    dict(gradp="superbee"),
    dict(limiter_k=2),
    dict(s_max=1, cfl_tau=0.3),
    dict(s_max=2),
    dict(s_max=4),
    dict(local_dtau=False),
    dict(realtime=False),
    dict(alpha_pi_p_row=False),
    dict(realtime=False, local_dtau=False, gradp="minmod", cfl_tau=0.9),
    dict(riemann="bassi"),
    dict(riemann="roe"),
    dict(gradp="split_minmod"),
    dict(gradp="split_superbee"),
]


@pytest.mark.parametrize("opts", OPTION_SETS, ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_option_matrix(opts):
    case = W.random_two_fluid(45, 21, ratio=200.0, c0=6.0, bc=("slip", "transmissive", "noslip", "slip"))
    for k, v in opts.items():
        setattr(case.options, k, v)
    assert_parity(run_both(case, steps=1, tol=-1.0, max_iters=5), case=case)


def test_convergence_terminated_dam_break():
    """Sec. 3.3.1 set-up (20x20, until the rho u and rho v residuals < 1e-3):
    same iteration count, same state."""
    case = W.dam_break_small()
    case.max_iters = 3000
    assert_parity(run_both(case, steps=1), case=case)


def test_hydrostatic_column_paper_setup():
    """Sec. 3.2 set-up (20x1, g along x, p = 0 at start, until rho u residual < 1e-5)."""
    case = W.hydrostatic_column_1d()
    case.max_iters = 5000
    assert_parity(run_both(case, steps=1), case=case)


@pytest.mark.parametrize("k", [1, 5])
@pytest.mark.parametrize("along", ["x", "y"])
def test_riemann_problem_pure_pseudo_time(k, along):
    """Sec. 3.1 set-up (real-time term off, global pseudo-time step, minmod on p)."""
    case = W.riemann_problem(k, 100, along=along)
    assert_parity(run_both(case, steps=1, tol=-1.0, max_iters=10), case=case)


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 17), (33, 1), (2, 2)])
def test_degenerate_grids(nx, ny):
    case = W.random_two_fluid(nx, ny, ratio=10.0, c0=3.0, velocity=0.01)
    assert_parity(run_both(case, steps=1, tol=-1.0, max_iters=3), case=case)


def test_not_converged_status():
    case = W.riemann_tank()
    res = run_both(case, steps=1, tol=1e-14, max_iters=3)
    got, ref, rc, its, st, oits, R, oR, R0, oR0 = res[0]
    assert rc == ac.AC_NOT_CONVERGED and its == 3 and st == oracle.NOT_CONVERGED
    assert_parity(res, case=case)


def test_nonfinite_restores_state():
    """A pseudo-CFL far beyond the stability limit makes the iteration blow
    up: the call reports AC_ERR_NONFINITE and leaves the state as it was."""
    case = W.random_two_fluid(32, 16, ratio=1000.0, c0=20.0)
    case.options.cfl_tau = 40.0
    t = ac.Tank.from_case(case)
    before = t.get_state()
    with pytest.raises(ac.ACError) as e:
        t.physical_step(case.dt, -1.0, 400)
    assert e.value.code == ac.AC_ERR_NONFINITE
    after = t.get_state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    t.close()


def test_state_roundtrip_and_resume_bitwise():
    """Checkpoint/resume: 3 steps == 1 step + get/set state + 2 steps, bitwise."""
    case = W.random_two_fluid(40, 24, ratio=100.0, c0=5.0)
    a = ac.Tank.from_case(case)
    for _ in range(3):
        a.physical_step(case.dt, -1.0, 4)
    full = a.get_state()
    b = ac.Tank.from_case(case)
    b.physical_step(case.dt, -1.0, 4)
    snap = b.get_state()
    b.close()
    c = ac.Tank.from_case(case)
    c.set_state(*snap)
    for _ in range(2):
        c.physical_step(case.dt, -1.0, 4)
    resumed = c.get_state()
    for x, y in zip(full, resumed):
        assert np.array_equal(x, y)
    s0 = case.state()
    d = ac.Tank.from_case(case)
    for x, y in zip(s0, d.get_state()):
        assert np.array_equal(x, y)
    for t in (a, c, d):
        t.close()


def test_runs_on_a_torch_stream():
    import torch
    case = W.random_two_fluid(40, 24, ratio=100.0, c0=5.0)
    s = torch.cuda.Stream()
    t = ac.Tank.from_case(case)
    t.set_stream(s.cuda_stream)
    rc, its = t.physical_step(case.dt, -1.0, 4)
    got = t.get_state()
    ref, *_ = oracle.physical_step(case, case.state(), tol=-1.0, max_iters=4)
    assert max(rel_errors(got, ref)) <= TOL
    # a step of 4 pseudo-iterations: 1 begin kernel + 4 x (3 stage sweeps + 1 end kernel)
    n0 = t.kernel_launches()
    t.physical_step(case.dt, -1.0, 4)
    assert t.kernel_launches() - n0 == 1 + 4 * 4
    t.close()


def test_step_before_state_is_an_error():
    t = ac.Tank(8, 8, 1.0, 1.0, 0.0, -9.81, 1e3, ("slip",) * 4)
    with pytest.raises(ac.ACError) as e:
        t.physical_step(1e-3, 1e-8, 10)
    assert e.value.code == ac.AC_ERR_STATE
    with pytest.raises(ac.ACError) as e:
        t.set_state(np.zeros(64), np.zeros(64), np.zeros(64), np.zeros(64))
    assert e.value.code == ac.AC_ERR_ARG
    bad = np.ones(64)
    bad[3] = math.nan
    with pytest.raises(ac.ACError) as e:
        t.set_state(np.ones(64), bad, np.zeros(64), np.zeros(64))
    assert e.value.code == ac.AC_ERR_NONFINITE
    t.close()


@pytest.mark.parametrize("riemann", ["bassi", "roe"])
@pytest.mark.parametrize("k", [1, 2, 5])
def test_riemann_problems_other_fluxes(riemann, k):
    """Sec. 3.1 set-up with the exact (Bassi) and Roe fluxes."""
    case = W.riemann_problem(k, 100)
    case.options.riemann = riemann
    assert_parity(run_both(case, steps=1, tol=-1.0, max_iters=10), case=case)


@pytest.mark.parametrize("order", [2, 3])
def test_bdf_steps_from_identical_history(order):
    """BDF2/BDF3 (Table BDF): each step starts GPU and oracle from the same
    state and the same older levels (ac_set_history / the oracle's history)."""
    case = W.random_two_fluid(37, 19, ratio=300.0, c0=8.0)
    case.options.bdf_order = order
    states = [case.state()]
    for step in range(4):
        older = [(s[0], s[1], s[2]) for s in states[::-1][1:3]]   # Q^{n-1}, Q^{n-2}
        ref, st, oits, oR, _ = oracle.physical_step(case, states[-1], tol=-1.0, max_iters=5, history=older)
        t = ac.Tank.from_case(case)
        t.set_state(*states[-1])
        for lvl, s_ in enumerate(states[::-1][1:3], start=1):
            if lvl == 2 and order < 2:
                break
            t.set_history(lvl, s_[0], s_[1], s_[2])
        t.physical_step(case.dt, -1.0, 5)
        got = t.get_state()
        t.close()
        errs = rel_errors(got, ref)
        assert max(errs) <= TOL, (step, errs)
        states.append(ref)


def test_bdf2_checkpoint_resume_bitwise():
    case = W.random_two_fluid(40, 24, ratio=100.0, c0=5.0)
    case.options.bdf_order = 2
    a = ac.Tank.from_case(case)
    for _ in range(4):
        a.physical_step(case.dt, -1.0, 4)
    full = a.get_state()
    b = ac.Tank.from_case(case)
    for _ in range(2):
        b.physical_step(case.dt, -1.0, 4)
    snap, h1, h2 = b.get_state(), b.get_history(1), b.get_history(2)
    b.close()
    c = ac.Tank.from_case(case)
    c.set_state(*snap)
    c.set_history(1, *h1)
    c.set_history(2, *h2)
    for _ in range(2):
        c.physical_step(case.dt, -1.0, 4)
    for x, y in zip(full, c.get_state()):
        assert np.array_equal(x, y)
    with pytest.raises(ac.ACError):
        a.get_history(3)
    a.close()
    c.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("mixed", 1e-6)])
def test_realtime_dt_from_cfl(precision, tol):
    """Sec. 2.2.4 global real-time step against the oracle, and +inf at rest."""
    case = W.random_two_fluid(45, 21, ratio=300.0, c0=8.0, velocity=0.3)
    t = ac.Tank.from_case(case, precision=precision)
    assert t.realtime_dt(0.45) == pytest.approx(oracle.realtime_dt(case, case.state(), 0.45), rel=tol)
    t.close()
    rest = W.hydrostatic_tank(32)
    t = ac.Tank.from_case(rest, precision=precision)
    assert t.realtime_dt(0.45) == math.inf
    t.close()


N_F64_VARIANTS = 8


@pytest.mark.parametrize("v", range(N_F64_VARIANTS))
@pytest.mark.parametrize("bc", [("periodic", "periodic", "slip", "noslip"), ("slip", "transmissive", "slip", "slip")])
def test_every_tile_variant(monkeypatch, v, bc):
    """Each compiled tile shape, forced in place of the autotuner's pick, on
    a grid with ragged tails in both directions for every shape."""
    monkeypatch.setenv("AC_TILE_F64", str(v))
    case = W.random_two_fluid(70, 45, ratio=1000.0, c0=20.0, bc=bc)
    t = ac.Tank.from_case(case)
    t.physical_step(case.dt, -1.0, 4)
    assert t.tile_shape()[3] == v
    got = t.get_state()
    t.close()
    ref, *_ = oracle.physical_step(case, case.state(), tol=-1.0, max_iters=4)
    errs = rel_errors(got, ref)
    assert max(errs) <= TOL, errs


def test_tile_shape_reported_after_the_first_step():
    case = W.random_two_fluid(40, 24, ratio=10.0, c0=5.0)
    t = ac.Tank.from_case(case)
    assert t.tile_shape()[3] == -1          # not tuned yet (AC_ERR_STATE)
    t.physical_step(case.dt, -1.0, 1)
    tx, ty, nt, v = t.tile_shape()
    assert v >= 0 and tx * ty >= nt > 0
    t.close()


def test_fp64_fma_probe_is_near_the_nominal_rate():
    """The FP64 FMA probe measures this part's rate: within a factor of two
    of the nominal 2 FMA lanes per SM at the current clock."""
    import torch
    v = ac.ac_probe_fp64_fma_tflops()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal_at_2ghz = 2 * 2 * sms * 2.0e9 / 1e12
    assert 0.5 * nominal_at_2ghz < v < 2.0 * nominal_at_2ghz, v
