"""Two single-tank configurations checked at their stated lengths on the GPU.

The Riemann tank 200x4 (rho 1000 | 1, p 1e5 | 0, at rest, transmissive in x,
periodic in y, dt 1e-4 s): its 20 physical steps, each ending on the 1e-8
residual drop or 500 pseudo-iterations (Alg. 1), the FP64 GPU path against the
FP64 oracle step by step (1e-11 per field, the same iteration counts and
status), and the mixed form within 1e-5 of the oracle after all 20 steps.  The
same tank in pure pseudo-time (Sec. 3.1 set-up: real-time term off, global
pseudo-time step, minmod on p) to tau = 1e-3 s, before the fastest wave leaves
the tank, against the exact solution of its Riemann problem sampled at x / tau
(the star states of the exact solver, Sec. 2.4.1, whose shock and rarefaction
relations the oracle pins check).

The hydrostatic two-fluid tank 256x256 at its stated 100 physical steps: both
forms stay at rest to 1e-10 m/s and the pressure keeps its kink, the slope
ratio water / air equal to the density ratio 1000.
"""
import numpy as np
import pytest

import oracle
from conftest import rel_errors
from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W
from test_gpu_parity import assert_parity, run_both

pytestmark = pytest.mark.gpu


def test_riemann_200x4_twenty_steps_against_oracle():
    case = W.riemann_tank()
    assert case.steps == 20
    assert_parity(run_both(case, steps=case.steps), case=case)


def test_riemann_200x4_twenty_steps_mixed_form():
    case = W.riemann_tank()
    st = case.state()
    t = ac.Tank.from_case(case, precision="mixed")
    for _ in range(case.steps):
        t.physical_step(case.dt, case.tol, case.max_iters)
        st, *_ = oracle.physical_step(case, st)
    got = t.get_state()
    t.close()
    assert max(rel_errors(got, st)) <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_riemann_200x4_pure_pseudo_time_against_exact_solution(precision):
    rp = W.riemann_tank()
    rp.options.realtime, rp.options.local_dtau, rp.options.gradp = False, False, "minmod"
    tau = 1e-3
    t = ac.Tank.from_case(rp, precision=precision)
    rc, n = t.pseudo_time_run(tau)
    q = t.get_state()
    t.close()
    assert rc == ac.AC_OK and n > 0
    xs = (np.arange(rp.nx) + 0.5) * (rp.lx / rp.nx) - 0.5
    left, right = [1000.0, 0.0, 0.0, 1e5], [1.0, 0.0, 0.0, 0.0]
    ex = np.array([oracle.bassi_sample(left, right, rp.beta, x / tau) for x in xs])
    sc = np.abs(ex).max(axis=0)
    l1_rho = np.abs(q[0][0] - ex[:, 0]).mean() / sc[0]
    l1_u = np.abs(q[1][0] / q[0][0] - ex[:, 1]).mean() / sc[1]
    l1_p = np.abs(q[3][0] - ex[:, 3]).mean() / sc[3]
    print(f"{precision}: {n} pseudo-iterations, relative L1 rho {l1_rho:.2e} u {l1_u:.2e} p {l1_p:.2e}")
    # a 200-cell second-order profile of a shock and a rarefaction: a few
    # cells of smearing at each wave
    assert l1_rho < 0.01 and l1_u < 0.1 and l1_p < 0.015
    # every row the same to round-off (the y direction is periodic and uniform)
    for f in range(4):
        assert np.abs(q[f] - q[f][0]).max() <= 1e-12 * max(np.abs(q[f]).max(), 1e-300)


def test_hydrostatic_256_hundred_steps_at_rest():
    case = W.hydrostatic_tank(256)
    assert case.steps == 100
    for precision in ("fp64", "mixed"):
        t = ac.Tank.from_case(case, precision=precision)
        for _ in range(case.steps):
            t.physical_step(case.dt, case.tol, case.max_iters)
        q = t.get_state()
        t.close()
        vmax = max(np.abs(q[1] / q[0]).max(), np.abs(q[2] / q[0]).max())
        assert vmax < 1e-10, (precision, vmax)
        col = q[3][:, case.nx // 2]
        sl = np.diff(col) / case.dy
        assert abs(sl[case.ny // 4] / sl[3 * case.ny // 4] - 1000.0) < 1e-6, precision
