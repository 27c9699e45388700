"""The allocation-free stage sweep (ac_stage_sweep_noalloc).

Callers that cannot allocate device memory (inside a memory pool they do not
own, a host that forbids allocation after start-up, a real-time loop) pass
their own device buffers; the sweep's scratch is a fixed array inside the
library.  Here the buffers come from torch, the caller.

Every case is checked against ac_physical_step of the same stage sequence
from the same state: relative L-infinity error <= 1e-11 per field, residual
norms to 1e-12 relative, and each is run on two calls (or two chains of
calls) in a row, the second on the first one's output.  This file is
collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from conftest import rel_errors
from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _reference_iteration(case, state):
    """One pseudo-iteration (all s_max stages) through ac_physical_step."""
    t = ac.Tank.from_case(case)
    t.set_state(*state)
    t.physical_step(case.dt, -1.0, 1)
    ref = t.get_state()
    R, _ = t.residual_norms()
    t.close()
    return ref, R


def _noalloc_iteration(case, opts, state, stream, dev):
    """The same pseudo-iteration as one allocation-free call per stage,
    chained through caller-owned buffers: stage s reads Q^{s-1} (the
    previous call's output) and Q^m."""
    import torch
    q0 = [torch.tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float64, device=dev) for a in state]
    norms = torch.full((4,), float("nan"), dtype=torch.float64, device=dev)
    prev = None
    for stage in range(1, case.options.s_max + 1):
        out = [torch.full_like(x, float("nan")) for x in q0]
        ac.ac_stage_sweep_noalloc(case.nx, case.ny, case.lx, case.ly, case.gx, case.gy, case.beta, case.bc,
                                  opts, stage, case.dt, None if prev is None else [x.data_ptr() for x in prev],
                                  [x.data_ptr() for x in q0], [x.data_ptr() for x in q0[:3]],
                                  [x.data_ptr() for x in out], norms.data_ptr() if stage == 1 else None,
                                  stream)
        prev = out
    torch.cuda.synchronize(dev)
    got = tuple(x.cpu().numpy().reshape(case.ny, case.nx) for x in prev)
    return got, norms.cpu().numpy()


@pytest.mark.parametrize("s_max,local_dtau", [(1, True), (3, True), (3, False)],
                         ids=["stage1_local_dtau", "three_stages_local_dtau", "three_stages_global_dtau"])
def test_noalloc_sweep_matches_physical_step_on_two_calls(s_max, local_dtau):
    import torch
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    case = W.random_two_fluid(70, 37, ratio=1000.0, c0=20.0, bc=("slip", "transmissive", "noslip", "slip"))
    case.options.s_max = s_max
    case.options.local_dtau = local_dtau
    opts = ac.options_from(case.options, "fp64")
    state = case.state()
    for call in range(2):
        ref, R = _reference_iteration(case, state)
        got, norms = _noalloc_iteration(case, opts, state, stream, dev)
        errs = rel_errors(got, ref)
        assert max(errs) <= 1e-11, (call, errs)
        assert np.allclose(norms, R, rtol=1e-12, atol=0.0), (call, norms, R)
        state = got


def test_noalloc_sweep_rejects_grids_beyond_its_scratch():
    """A grid larger than the fixed scratch is refused before any field
    pointer is read; the pointers here are NULL, which would be refused too
    if the size check were ever skipped, so nothing can be launched."""
    opts = ac.ac_default_options()
    with pytest.raises(ac.ACError) as e:
        ac.ac_stage_sweep_noalloc(4096, 4096, 1.0, 1.0, 0.0, -9.81, 1e3, ("slip",) * 4, opts, 1, 1e-3,
                                  None, [0, 0, 0, 0], [0, 0, 0], [0, 0, 0, 0], None, 0)
    assert e.value.code == ac.AC_ERR_ARG
    assert "scratch holds at most" in str(e.value)
