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


def field_scales(state):
    """Per-field scale for relative errors.  rho and p: max |field|.  The
    momentum is a vector: both components are measured against the largest
    momentum magnitude max |rho u|, floored at max(rho) * 1e-3 m/s so that a
    fluid at rest (round-off momenta) is compared against a physical scale
    rather than noise."""
    import numpy as np
    rho = np.abs(state[0]).max()
    mom = float(np.sqrt(np.asarray(state[1]) ** 2 + np.asarray(state[2]) ** 2).max())
    mom = max(mom, 1e-3 * rho)
    return [float(rho), mom, mom, max(float(np.abs(state[3]).max()), 1e-12)]


def rel_errors(got, ref):
    import numpy as np
    sc = field_scales(ref)
    return [float(np.abs(np.asarray(g) - np.asarray(r)).max() / s) for g, r, s in zip(got, ref, sc)]


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
