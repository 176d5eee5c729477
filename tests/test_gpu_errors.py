"""Failure detection on the GPU without a fault: a bounded device-side wait that expires.

The summation and reduced-basis kernels give up on any mbarrier wait after a time limit, latch
FEW_ERR_TIMEOUT in the context and wind down.  few_selftest_wait_expiry queues a kernel whose
one wait can never be satisfied (nothing arrives on its barrier and no copy is in flight), with
a short limit; the latch must report the timeout once, clear, and leave the context usable.
"""
import numpy as np
import pytest

from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W
from tests.gpu_common import to_host

pytestmark = pytest.mark.gpu


def test_expired_wait_latches_timeout_once(gpu_ctx):
    import time
    import torch
    assert gpu_ctx.sync_status() == F.FEW_OK
    t0 = time.perf_counter()
    F.few_selftest_wait_expiry(gpu_ctx.handle, 1000, RT.current_stream())
    assert gpu_ctx.sync_status() == F.FEW_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 1.0  # the 1 ms limit, not the 2 s default
    assert gpu_ctx.sync_status() == F.FEW_OK  # the latch is cleared by reading it
    # the context still works: a waveform afterwards is computed and identical to one before
    w = W.tiny_inputs(11, K=8, n_samples=3000)
    tr = RT.from_inputs(gpu_ctx, w)
    a = to_host(RT.waveform_inputs(gpu_ctx, tr, w, F.FEW_MIXED))
    F.few_selftest_wait_expiry(gpu_ctx.handle, 200, RT.current_stream())
    b = to_host(RT.waveform_inputs(gpu_ctx, tr, w, F.FEW_MIXED))
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_ERR_TIMEOUT
    np.testing.assert_array_equal(a, b)
    assert gpu_ctx.sync_status() == F.FEW_OK
    tr.release()


def test_selftest_rejects_bad_limits(gpu_ctx):
    for limit in (0, 2000001):
        with pytest.raises(F.FewError) as e:
            F.few_selftest_wait_expiry(gpu_ctx.handle, limit, RT.current_stream())
        assert e.value.status == F.FEW_ERR_INVALID_ARG
    assert gpu_ctx.sync_status() == F.FEW_OK
