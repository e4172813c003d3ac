import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def small_gauge():
    """4^4 gauge field of the plain FP64 workload: exp(i 0.3 H), no smearing."""
    import synth
    return synth.gauge((4, 4, 4, 4), 0.3, 0, 0.1, seed=1)
