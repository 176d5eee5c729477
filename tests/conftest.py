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


@pytest.fixture(scope="session")
def gpu_ctx():
    """One library context on cuda:0 for the whole GPU test session."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_04582_gb300 import _build
    from paper_2104_04582_gb300.runtime import Context
    _build.build()
    torch.cuda.init()
    ctx = Context(0)
    yield ctx
    ctx.close()
