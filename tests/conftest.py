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


def pytest_terminal_summary(terminalreporter):
    """The flagged closest-hit mismatches (ties, edges, order flips) of every parity
    comparison of the run, shown even with -q."""
    mod = sys.modules.get("tests.parity")
    if mod is None or not getattr(mod, "REPORTS", None):
        return
    terminalreporter.write_sep("-", "closest-hit parity: flagged mismatches per comparison")
    for label, line in mod.REPORTS:
        terminalreporter.write_line(f"{label}: {line}")
