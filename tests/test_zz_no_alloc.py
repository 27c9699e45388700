"""The allocation-free stage sweep (ac_stage_sweep_noalloc).

Callers that cannot allocate device memory (inside a memory pool they do not
own, a host that forbids allocation after start-up, a real-time loop) pass
their own device buffers; the sweep's scratch is a fixed array inside the
library.  Here the buffers come from torch, the caller.

Two calls in a row, the second on the first one's output, each checked
against ac_physical_step (one pseudo-iteration of one stage) from the same
state: relative L-infinity error <= 1e-11 per field, residual norms to
1e-12 relative.  This file is collected last so that a run stopping at the
first failure has run every other test before it.
"""
import numpy as np
import pytest

from conftest import rel_errors
from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_sweep_matches_physical_step_on_two_calls():
    import torch
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    case = W.random_two_fluid(70, 37, ratio=1000.0, c0=20.0, bc=("slip", "transmissive", "noslip", "slip"))
    case.options.s_max = 1   # one pseudo-iteration = one stage-1 sweep
    opts = ac.options_from(case.options, "fp64")
    state = case.state()
    for call in range(2):
        t = ac.Tank.from_case(case)
        t.set_state(*state)
        t.physical_step(case.dt, -1.0, 1)
        ref = t.get_state()
        R, _ = t.residual_norms()
        t.close()

        q0 = [torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device=dev) for a in state]
        qout = [torch.full_like(x, float("nan")) for x in q0]
        norms = torch.full((4,), float("nan"), dtype=torch.float64, device=dev)
        ac.ac_stage_sweep_noalloc(case.nx, case.ny, case.lx, case.ly, case.gx, case.gy, case.beta, case.bc,
                                  opts, 1, case.dt, None, [x.data_ptr() for x in q0],
                                  [x.data_ptr() for x in q0[:3]], [x.data_ptr() for x in qout],
                                  norms.data_ptr(), stream)
        torch.cuda.synchronize(dev)
        got = tuple(x.cpu().numpy().reshape(case.ny, case.nx) for x in qout)
        errs = rel_errors(got, ref)
        assert max(errs) <= 1e-11, (call, errs)
        assert np.allclose(norms.cpu().numpy(), R, rtol=1e-12, atol=0.0), (call, norms, R)
        state = got


def test_noalloc_sweep_rejects_grids_beyond_its_scratch():
    opts = ac.ac_default_options()
    with pytest.raises(ac.ACError) as e:
        ac.ac_stage_sweep_noalloc(4096, 4096, 1.0, 1.0, 0.0, -9.81, 1e3, ("slip",) * 4, opts, 1, 1e-3,
                                  None, [1, 1, 1, 1], [1, 1, 1], [1, 1, 1, 1], 0, 0)
    assert e.value.code == ac.AC_ERR_ARG
    assert "scratch holds at most" in str(e.value)
