import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU oracle run")


def cfl_dt(cp, dmin, cfl=0.3):
    """Time step from Eq. (5): dt = CFL * min(d) / max(cp)."""
    return cfl * dmin / float(np.max(cp))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def trace_errors(gpu, ref, floor_frac=1e-3):
    """Per-trace relative L2 error with the floor of the reading for
    near-zero traces: ||g - o|| / max(||o||, floor_frac * max_r ||o_r||),
    per component.  Returns the [4][n_rcv] array of errors."""
    g = np.asarray(gpu, np.float64)
    o = np.asarray(ref, np.float64)
    diff = np.linalg.norm(g - o, axis=-1)
    norm = np.linalg.norm(o, axis=-1)
    floor = floor_frac * norm.max(axis=1, keepdims=True)
    den = np.maximum(norm, floor)
    den = np.where(den > 0, den, 1.0)
    return diff / den


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
