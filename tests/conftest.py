import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def mht_lib():
    """Builds libmht.so in-tree if its sources changed, then loads it."""
    from paper_2605_21828_gb300 import build as bld
    bld.build_library()
    from paper_2605_21828_gb300 import _lib
    return _lib.load()
