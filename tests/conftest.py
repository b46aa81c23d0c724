import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def fnpf():
    """The ctypes binding of libfnpf.so, building the library in-tree if needed."""
    from paper_2506_09435_gb300 import build
    build.build()
    from paper_2506_09435_gb300 import fnpf as F
    return F
