import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def tiny_chain():
    """The tiny configuration: M=12, d=3, b_k = min(3^k, 3^(12-k), 16), unskewed Haar sites."""
    import gen

    w = gen.WORKLOADS["tiny"]
    b, ts, _ = gen.mps_tensors(w.M, w.d, w.chi, base_seed=w.base_seed, skew=w.skew)
    return b, ts


@pytest.fixture(scope="session")
def tiny_brute(tiny_chain):
    import oracle

    b, ts = tiny_chain
    return oracle.brute_force(b, ts)
