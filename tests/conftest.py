import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def oracle():
    from oracle import oracle as o
    o.build()
    return o


def build_lib():
    import __graft_entry__
    __graft_entry__._build_module().build()


def _gpu_ctx(prec):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_lib()
    import paper_1604_01814_gb300 as lgf
    ctx = lgf.Context(prec)
    ctx.table_build(48)
    return ctx


@pytest.fixture(scope="session")
def ctx64():
    c = _gpu_ctx("f64")
    yield c
    c.close()


@pytest.fixture(scope="session")
def ctx32():
    c = _gpu_ctx("f32")
    yield c
    c.close()


def rel_linf(got, ref):
    """Relative L-infinity error: max |got - ref| / max |ref| over all compared values."""
    import numpy as np
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))
