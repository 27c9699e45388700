import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(x) for x in line.split()])
    return rows


MOMENTUM_FLOOR = 1e-3   # m/s: momentum scales are at least max(rho) times this


def field_scales(state, floor=True):
    """Per-field scale for relative errors: every field, each momentum
    component included, against its own largest magnitude.  With `floor`,
    the momentum scales are at least max(rho) * MOMENTUM_FLOOR, so that a
    fluid at rest (round-off momenta) is compared against a physical scale
    rather than noise; without it only a zero field is replaced by 1e-300."""
    import numpy as np
    rho = float(np.abs(state[0]).max())
    mom = [float(np.abs(state[k]).max()) for k in (1, 2)]
    if floor:
        mom = [max(m, MOMENTUM_FLOOR * rho) for m in mom]
    else:
        mom = [max(m, 1e-300) for m in mom]
    return [rho, mom[0], mom[1], max(float(np.abs(state[3]).max()), 1e-12)]


def rel_errors(got, ref, floor=True):
    import numpy as np
    sc = field_scales(ref, floor)
    return [float(np.abs(np.asarray(g) - np.asarray(r)).max() / s) for g, r, s in zip(got, ref, sc)]


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
