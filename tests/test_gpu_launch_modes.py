"""The launch mode does not change a number.

A physical step runs as one graph launch (device-driven WHILE loop, kernels
with programmatic dependencies), as a host-driven loop (AC_LAUNCH=host), with
plain launches (AC_PDL=0), or one iteration at a time with per-stage events
(profiling).  All four give bit-identical states, iteration counts and
residual norms, in both precisions and for the batch.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2108_08769_gb300 import ac
from paper_2108_08769_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2108_08769_gb300 import ac, workloads as W
out = {}
for prec in ("fp64", "mixed"):
    case = W.random_two_fluid(70, 45, ratio=1000.0, c0=20.0)
    t = ac.Tank.from_case(case, precision=prec)
    rc, its = t.physical_step(case.dt, 1e-3, 40)
    R, R0 = t.residual_norms()
    out[prec] = {"its": its, "R": list(R), "state": [a.tolist() for a in t.get_state()]}
    t.close()
cases = W.batched_tanks(count=4, nmin=20, nmax=60, seed=7)
b = ac.Batch.from_cases(cases)
rc, its, st = b.physical_step(1e-3, -1.0, 6)
out["batch"] = {"its": its, "state": [[a.tolist() for a in b.get_state(k)] for k in range(len(cases))]}
b.close()
json.dump(out, open(sys.argv[2], "w"))
'''


def run_child(tmp_path, name, env_extra):
    script = tmp_path / "child.py"
    script.write_text(CHILD)
    out = tmp_path / f"{name}.json"
    env = dict(os.environ)
    # every process tunes on its own: pin the variants so that all modes run
    # the same kernels
    env.update({"AC_TILE": "0", "AC_TILE_F64": "0", "AC_BATCH_TILE": "0"})
    env.update(env_extra)
    subprocess.run([sys.executable, str(script), ROOT, str(out)], env=env, check=True, timeout=600)
    return json.load(open(out))


def test_graph_host_loop_and_plain_launches_agree(tmp_path):
    base = run_child(tmp_path, "graph", {})
    for name, extra in [("host", {"AC_LAUNCH": "host"}), ("nopdl", {"AC_PDL": "0"})]:
        other = run_child(tmp_path, name, extra)
        assert other == base, name


def test_profiling_mode_agrees_with_the_graph(monkeypatch):
    monkeypatch.setenv("AC_TILE", "0")
    case = W.random_two_fluid(70, 45, ratio=1000.0, c0=20.0)
    results = []
    for prof in (False, True):
        t = ac.Tank.from_case(case, precision="mixed")
        t.set_profiling(prof)
        rc, its = t.physical_step(case.dt, 1e-3, 40)
        R, _ = t.residual_norms()
        results.append((its, R, t.get_state()))
        t.close()
    (i0, r0, s0), (i1, r1, s1) = results
    assert i0 == i1 and np.array_equal(r0, r1)
    for x, y in zip(s0, s1):
        assert np.array_equal(x, y)


LOG_CHILD = r'''
import sys
sys.path.insert(0, sys.argv[1])
from paper_2108_08769_gb300 import ac, workloads as W
case = W.random_two_fluid(16, 8)
t = ac.Tank.from_case(case)
t.physical_step(case.dt, -1.0, 3)
t.physical_step(case.dt, -1.0, 2)
t.close()
cases = W.batched_tanks(count=3, nmin=16, nmax=24, seed=3)
b = ac.Batch.from_cases(cases)
b.physical_step(1e-3, -1.0, 4)
b.close()
'''


def test_ac_log_prints_one_line_per_step(tmp_path):
    """AC_LOG=1: every physical step, single tank or batch, prints one line
    on stderr with its iterations, status and norms."""
    script = tmp_path / "log_child.py"
    script.write_text(LOG_CHILD)
    r = subprocess.run([sys.executable, str(script), ROOT], env=dict(os.environ, AC_LOG="1"),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    single = [l for l in r.stderr.splitlines() if l.startswith("ac_physical_step:")]
    batch = [l for l in r.stderr.splitlines() if l.startswith("ac_batch_physical_step:")]
    assert len(single) == 2 and len(batch) == 1, r.stderr[-2000:]
    assert "16x8 fp64 rc=0 iters=3 " in single[0] and "iters=2 " in single[1]
    assert "R0=(" in single[0] and "R=(" in single[0]
    assert "3 tanks rc=0 iters=4..4" in batch[0]
    quiet = subprocess.run([sys.executable, str(script), ROOT], env=dict(os.environ, AC_LOG="0"),
                           capture_output=True, text=True, timeout=600)
    assert quiet.returncode == 0 and "ac_physical_step:" not in quiet.stderr
