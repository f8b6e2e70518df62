import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session", autouse=True)
def _built_library():
    """Build libdmrgc.so once if it is missing (nvcc cross-compiles without a GPU)."""
    lib = os.path.join(ROOT, "paper_2207_05612_gb300", "lib", "libdmrgc.so")
    if not os.path.exists(lib):
        from paper_2207_05612_gb300 import build
        build.build()
    yield
