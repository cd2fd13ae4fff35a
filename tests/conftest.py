"""Shared pytest configuration.

Tests that need a CUDA device carry ``@pytest.mark.gpu``; everything else runs on the
CPU (the FP64 oracle, its pins, host-side logic, ABI loading and argument checks).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
