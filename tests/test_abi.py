"""The C ABI library loads and exports every entry point include/*.h
declares; argument validation happens on the host before any CUDA call."""
import glob
import os
import re
import subprocess

import pytest

from conftest import ROOT
from paper_2108_08769_gb300 import ac


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(ac_\w+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_header_declares_the_binding_exports():
    assert declared_symbols() == set(ac.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = ac.load().__dict__.get("_name") or ac.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = declared_symbols() - exported
    assert not missing, missing
    L = ac.load()
    for name in declared_symbols():
        assert hasattr(L, name)


def test_default_options_and_beta_helper():
    o = ac.ac_default_options()
    assert (o.rk_stages, o.gradp, o.limiter_k, o.local_dtau, o.realtime) == (3, 0, 1, 1, 1)
    assert o.cfl_tau == pytest.approx(0.45)
    assert ac.ac_beta_from_speed(20.0, 1000.0) == pytest.approx(4e5)


@pytest.mark.parametrize("kw,fragment", [
    (dict(nx=0), "nx, ny"),
    (dict(beta=-1.0), "beta"),
    (dict(bc=("periodic", "slip", "slip", "slip")), "periodic"),
    (dict(lx=0.0), "lx"),
    (dict(nx=65536, ny=32769), "2^31"),
])
def test_create_rejects_bad_arguments_before_touching_the_gpu(kw, fragment):
    args = dict(nx=8, ny=8, lx=1.0, ly=1.0, gx=0.0, gy=-9.81, beta=1e3, bc=("slip",) * 4)
    args.update(kw)
    with pytest.raises(ac.ACError) as e:
        ac.Tank(**args)
    assert e.value.code == ac.AC_ERR_ARG
    assert fragment in str(e.value)


def test_create_rejects_bad_options():
    o = ac.ac_default_options()
    o.rk_stages = 7
    with pytest.raises(ac.ACError) as e:
        ac.Tank(8, 8, 1.0, 1.0, 0.0, -9.81, 1e3, ("slip",) * 4, options=o)
    assert e.value.code == ac.AC_ERR_ARG


def _tank_stub(nx=8, ny=8, beta=1e3, bc=("slip",) * 4, **opt):
    from types import SimpleNamespace
    from paper_2108_08769_gb300 import workloads as W
    return SimpleNamespace(nx=nx, ny=ny, lx=1.0, ly=1.0, gx=0.0, gy=-9.81, beta=beta, bc=bc,
                           options=W.Options(**opt))


@pytest.mark.parametrize("cases,fragment", [
    ([], "1..65535"),
    ([_tank_stub(), _tank_stub(nx=0)], "tank 1: invalid grid"),
    ([_tank_stub(beta=0.0)], "beta"),
    ([_tank_stub(bc=("slip", "slip", "periodic", "slip"))], "periodic"),
    ([_tank_stub(local_dtau=False)], "local pseudo-time step"),
    ([_tank_stub(nx=46341, ny=46341)], "2^31"),
    ([_tank_stub(nx=32768, ny=32768), _tank_stub(nx=32768, ny=32768), _tank_stub()], "2^31"),
])
def test_batch_create_rejects_bad_arguments_before_touching_the_gpu(cases, fragment):
    """ac_batch_create checks every tank and the batch's total size before
    any device call (no GPU here)."""
    if not cases:
        with pytest.raises(ac.ACError) as e:
            ac._check(ac.load().ac_batch_create(0, None, None, None, None, ac.C.byref(ac.C.c_void_p())))
    else:
        with pytest.raises(ac.ACError) as e:
            ac.Batch(cases)
    assert e.value.code == ac.AC_ERR_ARG
    assert fragment in str(e.value)
