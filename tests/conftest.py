import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def qlib():
    """The built libqaoa binding (compiled in-tree if missing or stale)."""
    from paper_2101_10296_gb300 import build
    build.build()
    from paper_2101_10296_gb300 import qaoa
    qaoa.lib()
    return qaoa
