"""Shared pytest configuration.

Markers:
  gpu   needs a CUDA device and the compiled CUDA library (run with -m gpu)
  slow  CPU tests that take more than a few seconds
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
