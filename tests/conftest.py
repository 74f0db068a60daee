import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture
def rng():
    return np.random.default_rng(12345)


_LIB_BUILT = {}


def built_library():
    """Builds liblorads.so in-tree (no-op when up to date) and loads it."""
    if "lib" not in _LIB_BUILT:
        from paper_2403_09133_gb300 import build as B
        from paper_2403_09133_gb300 import lorads as L
        B.build()
        _LIB_BUILT["lib"] = L.load_library()
    return _LIB_BUILT["lib"]


@pytest.fixture(scope="session")
def lib():
    return built_library()


@pytest.fixture(scope="session")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_library()
    return torch
