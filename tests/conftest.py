import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size cases")


@pytest.fixture(scope="session")
def gwlib():
    """The C-ABI library, built in-tree for sm_103a if missing or stale."""
    from paper_1911_05633_gb300 import build, gw
    build.build()
    return gw.load_library()
