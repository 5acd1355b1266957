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
def wl1():
    import synthetic
    return synthetic.make(1)


@pytest.fixture(scope="session")
def wl2_small():
    """Config-2 scene and materials at 96x96: every ray type, oracle-sized."""
    import synthetic
    return synthetic.make(2, res=96)
