"""Mixed form (FP32 sweep; FP64 time levels, reference pressure and residual
sums) against FP64, element by element, through the C ABI.

Bar: relative L-infinity error <= 1e-5 per field after physical steps with a
fixed number of pseudo-iterations from an identical input state.  Every
field is measured against its own largest magnitude, each momentum
component separately; momentum scales are floored at max(rho) * 1e-3 m/s
so that a fluid at rest compares against a physical scale (the full-size
moving-flow cases below also pass unfloored).  Small cases compare with the
FP64 oracle; full-size cases with the FP64 GPU path, which itself matches the
oracle to 1e-11 (test_gpu_parity.py).
"""
import numpy as np
import pytest

import oracle
from conftest import rel_errors
from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


def gpu_run(case, precision, steps=1, iters=10, tol=-1.0, norms=False):
    t = ac.Tank.from_case(case, precision=precision)
    its, R0s = [], []
    for _ in range(steps):
        rc, n = t.physical_step(case.dt, tol, iters)
        its.append(n)
        R0s.append(t.residual_norms()[1])
    out = t.get_state()
    R, R0 = t.residual_norms()
    t.close()
    if norms:
        return out, its, R, np.array(R0s)
    return out, its, R


def oracle_run(case, steps=1, iters=10):
    s = case.state()
    for _ in range(steps):
        s, *_ = oracle.physical_step(case, s, tol=-1.0, max_iters=iters)
    return s


def check(got, ref, tol=TOL, floor=True):
    errs = rel_errors(got, ref, floor)
    assert max(errs) <= tol, errs
    return errs


def test_hydrostatic_tank_stays_balanced():
    case = W.hydrostatic_tank(64)
    got, _, R = gpu_run(case, "mixed", iters=40)
    ref = oracle_run(case, iters=40)
    check(got, ref)
    # the reference split keeps the rest state exact in FP32
    assert np.abs(got[1]).max() < 1e-9 and np.abs(got[2]).max() < 1e-9


@pytest.mark.parametrize("bc", [("slip",) * 4, ("noslip", "slip", "slip", "noslip"),
                                ("periodic", "periodic", "slip", "slip"),
                                ("slip", "transmissive", "transmissive", "slip"),
                                ("periodic",) * 4])
def test_random_two_fluid_against_oracle(bc):
    case = W.random_two_fluid(45, 21, ratio=1000.0, c0=20.0, bc=bc,
                              gy=0.0 if bc[2] == "periodic" else -9.81)
    got, _, _ = gpu_run(case, "mixed", iters=8)
    ref = oracle_run(case, iters=8)
    check(got, ref)


@pytest.mark.parametrize("opts", [dict(gradp="minmod"), dict(local_dtau=False), dict(s_max=2),
                                  dict(limiter_k=2), dict(realtime=False, cfl_tau=0.3),
                                  dict(riemann="bassi"), dict(riemann="roe"), dict(gradp="split_minmod")],
                         ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_options_against_oracle(opts):
    case = W.random_two_fluid(37, 19, ratio=100.0, c0=6.0)
    for k, v in opts.items():
        setattr(case.options, k, v)
    got, _, _ = gpu_run(case, "mixed", iters=6)
    ref = oracle_run(case, iters=6)
    check(got, ref)


def test_riemann_tank_against_oracle():
    case = W.riemann_tank()
    got, _, _ = gpu_run(case, "mixed", iters=60)
    ref = oracle_run(case, iters=60)
    check(got, ref)


def test_water_column_levels_accumulate_over_steps():
    """Three physical steps: the FP64 level absorbs each step's FP32
    increment, so the error does not grow with the step count."""
    case = W.water_column(128, 64)
    got, _, _ = gpu_run(case, "mixed", steps=3, iters=30)
    ref = oracle_run(case, steps=3, iters=30)
    check(got, ref)


def test_dam_break_small_paper_setup_against_oracle():
    case = W.dam_break_small()
    got, _, _ = gpu_run(case, "mixed", iters=200)
    ref = oracle_run(case, iters=200)
    check(got, ref)


def test_rayleigh_taylor_256x1024_against_fp64_gpu():
    case = W.rayleigh_taylor(256, 1024)
    mixed, _, _ = gpu_run(case, "mixed", iters=20)
    f64, _, _ = gpu_run(case, "fp64", iters=20)
    check(mixed, f64)


def test_rayleigh_taylor_2048x8192_against_fp64_gpu():
    """The full 2048x8192 grid, once the flow moves: mixed vs FP64 GPU on
    every cell after five physical steps of 20 pseudo-iterations, each
    momentum component against its own maximum, with no floor."""
    case = W.rayleigh_taylor(2048, 8192)
    mixed, _, _ = gpu_run(case, "mixed", steps=5, iters=20)
    f64, _, _ = gpu_run(case, "fp64", steps=5, iters=20)
    check(mixed, f64, floor=False)


def test_water_column_1024x512_moving_flow_per_component():
    """The 1024x512 collapsing column after three physical steps of 30
    pseudo-iterations: the column edge carries a pressure jump of the size
    of the hydrostatic head, and the air beside it moves; the pressure is
    carried as an FP32 increment over its FP64 level and each face is solved
    relative to the levels' mean, so FP32 holds only increments and
    cell-to-cell jumps.  Each momentum component against its own maximum,
    no floor.  (Within the first few pseudo-iterations after the release the
    pressure increment at the column edge is itself of the size of the head,
    and its FP32 rounding carries into rho v there, ~3e-5 of max |rho v|
    after one step of 20 iterations; it decays as the pseudo-time iteration
    converges.)"""
    case = W.water_column(1024, 512)
    mixed, _, _ = gpu_run(case, "mixed", steps=3, iters=30)
    f64, _, _ = gpu_run(case, "fp64", steps=3, iters=30)
    check(mixed, f64, floor=False)


@pytest.mark.parametrize("case_fn", [lambda: W.water_column(1024, 512), W.riemann_tank, W.dam_break_small,
                                     lambda: W.rayleigh_taylor(512, 2048)],
                         ids=["water_column_1024x512", "riemann_tank", "dam_break_small", "rayleigh_taylor_512x2048"])
def test_first_residual_norms_match_fp64(case_fn):
    """Alg. 1's residual norms R0 (the stage-1 bracket's RMS at the first
    pseudo-iteration of each step, summed in FP64 in both forms) agree with
    the FP64 path to 2e-6 relative over three steps, for every field whose
    FP64 norm is above round-off (a field at rest has R0 ~ 1e-13 in FP64 and
    exactly 0 in the mixed form)."""
    case = case_fn()
    _, _, _, m0 = gpu_run(case, "mixed", steps=3, iters=20, norms=True)
    _, _, _, f0 = gpu_run(case, "fp64", steps=3, iters=20, norms=True)
    live = f0 > 1e-9 * f0.max()
    rel = np.abs(m0 - f0)[live] / f0[live]
    assert rel.max() <= 2e-6, (rel.max(), m0, f0)
    assert np.all(np.abs(m0[~live]) <= 1e-9 * f0.max())


@pytest.mark.parametrize("tol", [1e-3, 1e-4])
def test_stopping_test_iteration_counts_match_fp64(tol):
    """With the stopping test on (Alg. 1, R <= tol R0), the mixed form stops
    within one pseudo-iteration of the FP64 form on every step of a moving
    two-fluid tank (the FP64 form needs 422-1196 iterations here), and on the
    first step of the Riemann tank at tol 1e-2.  Below R/R0 ~ 1e-6 the FP32
    state's own round-off sets a floor the mixed form cannot pass."""
    case = W.random_two_fluid(45, 21, ratio=1000.0, c0=20.0)
    _, mi, _ = gpu_run(case, "mixed", steps=3, iters=3000, tol=tol)
    _, fi, _ = gpu_run(case, "fp64", steps=3, iters=3000, tol=tol)
    assert max(fi) < 3000
    assert all(abs(a - b) <= 1 for a, b in zip(mi, fi)), (mi, fi)
    rt = W.riemann_tank()
    _, mi, _ = gpu_run(rt, "mixed", steps=1, iters=3000, tol=1e-2)
    _, fi, _ = gpu_run(rt, "fp64", steps=1, iters=3000, tol=1e-2)
    assert fi[0] < 3000 and abs(mi[0] - fi[0]) <= 1, (mi, fi)


def test_state_roundtrip_mixed():
    case = W.water_column(64, 32)
    t = ac.Tank.from_case(case, precision="mixed")
    got = t.get_state()
    for a, b in zip(got[:3], case.state()[:3]):
        assert np.array_equal(a, b)
    assert np.abs(got[3] - case.p).max() <= 1e-6 * max(np.abs(case.p).max(), 1.0)
    t.close()


def test_nonfinite_restores_state_mixed():
    case = W.random_two_fluid(32, 16, ratio=1000.0, c0=20.0)
    case.options.cfl_tau = 40.0
    t = ac.Tank.from_case(case, precision="mixed")
    before = t.get_state()
    with pytest.raises(ac.ACError) as e:
        t.physical_step(case.dt, -1.0, 400)
    assert e.value.code == ac.AC_ERR_NONFINITE
    after = t.get_state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    t.close()


def test_converged_step_close_to_oracle():
    """With the stopping test on, both forms stop near the same iteration
    and land on the same converged state within the tolerance's reach."""
    case = W.riemann_tank()
    got, its, _ = gpu_run(case, "mixed", iters=500, tol=1e-6)
    ref, st, oits, *_ = oracle.physical_step(case, case.state(), tol=1e-6, max_iters=500)
    assert abs(its[0] - oits) <= max(2, oits // 20), (its, oits)
    check(got, ref, tol=1e-4)


@pytest.mark.parametrize("order", [2, 3])
def test_bdf_levels_against_oracle(order):
    """Four physical steps with BDF2/BDF3: the mixed form carries the older
    levels as FP32 differences to the FP64 level; against the oracle run
    with its explicit history."""
    case = W.water_column(96, 48)
    case.options.bdf_order = order
    t = ac.Tank.from_case(case, precision="mixed")
    states = [case.state()]
    for step in range(4):
        t.physical_step(case.dt, -1.0, 12)
        older = [(s[0], s[1], s[2]) for s in states[::-1][1:3]]   # Q^{n-1}, Q^{n-2}
        ref, *_ = oracle.physical_step(case, states[-1], tol=-1.0, max_iters=12, history=older)
        states.append(ref)
    check(t.get_state(), states[-1])
    t.close()


N_MIXED_VARIANTS = 22


@pytest.mark.parametrize("v", range(N_MIXED_VARIANTS))
@pytest.mark.parametrize("bc", [("periodic", "periodic", "slip", "noslip"), ("slip", "transmissive", "slip", "slip"),
                                ("slip", "slip", "transmissive", "slip")],
                         ids=["periodic_x_walls_y", "walls_transmissive_x", "reference_off"])
def test_every_tile_variant_against_oracle(monkeypatch, v, bc):
    """Each compiled tile shape and load scheme (direct or prefetched),
    forced in place of the autotuner's pick, on a grid with ragged tails in
    both directions; the first two boundary sets use the hydrostatic
    reference, the third runs without it."""
    monkeypatch.setenv("AC_TILE", str(v))
    case = W.random_two_fluid(70, 45, ratio=1000.0, c0=20.0, bc=bc)
    t = ac.Tank.from_case(case, precision="mixed")
    t.physical_step(case.dt, -1.0, 6)
    assert t.tile_shape()[3] == v
    got = t.get_state()
    t.close()
    check(got, oracle_run(case, iters=6))


STRIP_VARIANTS = [16, 18]   # column-strip sweeps, 64- and 256-row strips


@pytest.mark.parametrize("v", STRIP_VARIANTS, ids=["strips_64", "strips_256"])
@pytest.mark.parametrize("opts", [dict(limiter_k=2), dict(realtime=False, cfl_tau=0.3), dict(local_dtau=False),
                                  dict(alpha_pi_p_row=False), dict(s_max=2), dict(s_max=4)],
                         ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_strip_sweep_options_against_oracle(monkeypatch, opts, v):
    """The column-strip sweep under every option it implements (the new
    pressure gradient and Backward-Euler), forced on a ragged grid whose
    strips have ghost columns on both sides."""
    monkeypatch.setenv("AC_TILE", str(v))
    case = W.random_two_fluid(61, 83, ratio=300.0, c0=10.0, bc=("slip", "noslip", "slip", "transmissive"))
    for name, value in opts.items():
        setattr(case.options, name, value)
    t = ac.Tank.from_case(case, precision="mixed")
    t.physical_step(case.dt, -1.0, 6)
    assert t.tile_shape()[3] == v
    got = t.get_state()
    t.close()
    check(got, oracle_run(case, iters=6))


EDGE_GRIDS = [(61, 83, ("slip", "slip", "periodic", "periodic"), 0.0),
              (45, 70, ("periodic", "periodic", "slip", "noslip"), -9.81),
              (29, 3, ("slip", "noslip", "slip", "slip"), -9.81),
              (33, 1, ("transmissive", "slip", "slip", "slip"), -9.81),
              (2, 2, ("slip", "slip", "slip", "slip"), -9.81)]


@pytest.mark.parametrize("v", [15, 16], ids=["strips_32", "strips_64"])
@pytest.mark.parametrize("grid", EDGE_GRIDS, ids=["61x83_periodic_y", "45x70_walls_y", "29x3", "33x1", "2x2"])
@pytest.mark.parametrize("opts", [dict(), dict(limiter_k=2)], ids=["default_options", "limiter_k=2"])
def test_strip_sweep_edge_rows_against_oracle(monkeypatch, v, grid, opts):
    """The column-strip sweep's three row loops (a strip's first four rows,
    the rows whose window holds tank rows only, the top strip's last rows) on
    grids where they meet the tank's edges: periodic y (ghost rows fold onto
    the other end, the top face's jump is the bottom one's), a ragged top
    strip (70 rows in 32-row strips), and tanks of 3, 1 and 2 rows, where the
    main loop has no row at all; with the default options (the instances that
    compile them in) and with another limiter (the general instance)."""
    nx, ny, bc, gy = grid
    monkeypatch.setenv("AC_TILE", str(v))
    case = W.random_two_fluid(nx, ny, ratio=300.0, c0=10.0, bc=bc, gy=gy)
    for name, value in opts.items():
        setattr(case.options, name, value)
    t = ac.Tank.from_case(case, precision="mixed")
    t.physical_step(case.dt, -1.0, 6)
    assert t.tile_shape()[3] == v
    got = t.get_state()
    t.close()
    check(got, oracle_run(case, iters=6))
