"""Shared pytest configuration.

Markers:
  gpu   needs a CUDA device and the compiled CUDA library (run with -m gpu)
  slow  CPU tests that take more than a few seconds
  scale GPU parity at full benchmark size against the oracle on every host
        core (minutes; part of -m gpu)
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and libgbbc.so")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")
    config.addinivalue_line("markers", "scale: full-size GPU parity against the multi-core oracle")


@pytest.fixture(scope="session")
def gb():
    """The CUDA library's binding, built for this machine (skips without a GPU)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2008_05718_gb300 import _build, gbbc
    _build.build()
    gbbc.load()
    return gbbc
