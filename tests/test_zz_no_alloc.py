"""few_waveform_noalloc, the allocation-free entry point, against few_waveform.

Some callers must not allocate once they are running -- a sampler or a real-time pipeline that
reserves all device memory at start-up, or code where cudaMalloc is not allowed on the call
path.  For them the library offers few_waveform_noalloc, which keeps its scratch in a fixed
device array inside the library.  These tests call it through the C ABI and check that two
calls in a row (different sizes, precisions and mode sets, so the second reuses the array the
first one filled) give what the allocating entry point gives, within the parity tolerances of
the other GPU tests, and that an oversized request is refused.

This file is collected last on purpose: if it fails, every other test has already run.
"""
import numpy as np
import pytest

from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W
from tests.gpu_common import FP64_REL_L2, MIXED_MISMATCH, rel_l2, to_host

pytestmark = pytest.mark.gpu


def _mismatch(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    d = a / np.linalg.norm(a) - b / np.linalg.norm(b)
    return float(0.5 * np.vdot(d, d).real)


def _both(ctx, tr, w, prec):
    """(allocating entry point, allocation-free entry point) outputs for one request."""
    import torch
    c64 = prec == F.FEW_MIXED
    ref = RT.alloc_out(w.n_samples, c64)
    got = RT.alloc_out(w.n_samples, c64)
    got.fill_(complex(np.nan, np.nan))
    s = RT.current_stream()
    F.few_waveform(ctx.handle, RT.request(tr, ref, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec,
                                          w.scale), s)
    F.few_waveform_noalloc(ctx.handle, RT.request(tr, got, w.n_samples, w.t0, w.dt, w.theta,
                                                  w.phi, prec, w.scale), s)
    torch.cuda.synchronize()
    assert ctx.sync_status() == F.FEW_OK
    return to_host(ref), to_host(got)


def _allocation_state(ctx):
    """(bytes the library context holds, free device bytes) -- both must stay put."""
    import torch
    in_use, _ = ctx.memory()
    return in_use, torch.cuda.mem_get_info()[0]


def test_noalloc_allocates_nothing(gpu_ctx):
    import torch
    w = W.config1()
    tr = RT.from_inputs(gpu_ctx, w)
    out = RT.alloc_out(w.n_samples, True)
    req = RT.request(tr, out, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_MIXED, w.scale)
    F.few_waveform_noalloc(gpu_ctx.handle, req, RT.current_stream())  # first call: set-up
    torch.cuda.synchronize()
    before = _allocation_state(gpu_ctx)
    for _ in range(3):
        F.few_waveform_noalloc(gpu_ctx.handle, req, RT.current_stream())
    torch.cuda.synchronize()
    assert _allocation_state(gpu_ctx) == before
    assert gpu_ctx.sync_status() == F.FEW_OK
    tr.release()


def test_noalloc_detector_frame(gpu_ctx):
    """Detector-frame (Sec. 2.A) requests take the same path and agree with few_waveform."""
    import torch
    w = W.config1()
    tr = RT.from_inputs(gpu_ctx, w)
    outs = []
    for fn in (F.few_waveform, F.few_waveform_noalloc):
        out = RT.alloc_out(w.n_samples, False)
        req = RT.request(tr, out, w.n_samples, w.t0, w.dt, 1.1, 0.4, F.FEW_FP64, w.scale,
                         frame=F.FEW_FRAME_SSB, theta_K=0.3, phi_K=2.0)
        fn(gpu_ctx.handle, req, RT.current_stream())
        outs.append(out)
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    assert rel_l2(to_host(outs[1]), to_host(outs[0])) <= FP64_REL_L2
    tr.release()


def test_noalloc_matches_waveform_on_two_calls_in_a_row(gpu_ctx):
    # call 1: the one-year 3843-mode workload in FP64 (fills most of the fixed array)
    w1 = W.config2()
    tr1 = RT.from_inputs(gpu_ctx, w1)
    ref1, got1 = _both(gpu_ctx, tr1, w1, F.FEW_FP64)
    assert np.all(np.isfinite(got1))
    assert rel_l2(got1, ref1) <= FP64_REL_L2
    # call 2: a smaller, different mode set in mixed precision, reusing the array
    w2 = W.config1()
    tr2 = RT.from_inputs(gpu_ctx, w2)
    ref2, got2 = _both(gpu_ctx, tr2, w2, F.FEW_MIXED)
    assert np.all(np.isfinite(got2))
    assert _mismatch(got2, ref2) <= MIXED_MISMATCH
    assert rel_l2(got2, ref2) <= 1e-6
    tr1.release()
    tr2.release()


def test_noalloc_refuses_requests_beyond_its_array(gpu_ctx):
    # the four-year workload needs ~24.5 MB of folded FP64 coefficients: more than the array
    # (and, mixed, ~190 MB of phase anchors)
    w = W.config5()
    tr = RT.from_inputs(gpu_ctx, w)
    out = RT.alloc_out(1000, False)
    with pytest.raises(F.FewError) as e:
        F.few_waveform_noalloc(gpu_ctx.handle, RT.request(tr, out, 1000, w.t0, w.dt, w.theta,
                                                          w.phi, F.FEW_FP64), RT.current_stream())
    assert e.value.status == F.FEW_ERR_LIMIT
    host = np.zeros(1000, dtype=np.complex128)
    with pytest.raises(F.FewError) as e:  # host output buffers are not accepted
        F.few_waveform_noalloc(gpu_ctx.handle, RT.request(tr, host, 1000, w.t0, w.dt, w.theta,
                                                          w.phi, F.FEW_FP64,
                                                          out_where=F.FEW_MEM_HOST), 0)
    assert e.value.status == F.FEW_ERR_INVALID_ARG
    assert gpu_ctx.sync_status() == F.FEW_OK
    tr.release()
