"""Shared pytest configuration.

Tests marked ``gpu`` need a GB300 and the compiled CUDA library; everything else runs on a
CPU-only machine (oracle pins, host planning logic, ABI symbol checks, gloo multi-process
checks of the sharded benchmark path).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")
