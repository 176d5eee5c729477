"""GPU tests of the batched path: many waveforms of uneven length and mode count in one persistent
summation launch, captured once in a CUDA graph and replayed.

* every waveform of a batch is bit-identical to the same request run alone (the per-sample
  summation order does not depend on the batch);
* graph replays are bit-identical; a batch with FEW_BATCH_REBUILD_SPLINES picks up new knot data;
* the 256-waveform batch workload (0.25-2 yr, K 50-150, power-selected 10-3843 modes) matches the
  oracle on sampled windows.
"""
import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W
from tests.gpu_common import FP64_REL_L2, MIXED_MISMATCH, oracle_threads, rel_l2, to_host

pytestmark = pytest.mark.gpu


def _mixed_set(seed=7):
    rng = np.random.default_rng(seed)
    ws = [W.config1(), W.tiny_inputs(3, K=9, n_samples=5000)]
    g = np.random.Generator(np.random.PCG64(seed))
    for k in range(4):
        T = float(g.uniform(0.02, 0.1)) * W.YEAR_S
        ws.append(W.subset_waveform(g, T, int(g.integers(12, 40)), float(rng.choice([5.0, 10.0, 15.0])),
                                    600, name=f"sub{k}"))
    return ws


def _alone(ctx, tr, w, prec):
    import torch
    out = RT.waveform_inputs(ctx, tr, w, prec)
    torch.cuda.synchronize()
    return to_host(out)


@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
def test_batch_equals_alone_bitwise(gpu_ctx, prec):
    import torch
    ws = _mixed_set()
    trs = [RT.from_inputs(gpu_ctx, w) for w in ws]
    c64 = prec == F.FEW_MIXED
    outs = [RT.alloc_out(w.n_samples, c64) for w in ws]
    reqs = [RT.request(tr, o, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec, w.scale)
            for tr, o, w in zip(trs, outs, ws)]
    b = F.few_batch_plan(gpu_ctx.handle, reqs)
    F.few_batch_run(gpu_ctx.handle, b, RT.current_stream())
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    first = [to_host(o) for o in outs]
    for o in outs:
        o.zero_()
    F.few_batch_run(gpu_ctx.handle, b, RT.current_stream())  # graph replay
    torch.cuda.synchronize()
    for w, tr, o, h in zip(ws, trs, outs, first):
        np.testing.assert_array_equal(to_host(o), h)
        np.testing.assert_array_equal(_alone(gpu_ctx, tr, w, prec), h)
    F.few_batch_release(gpu_ctx.handle, b)
    # one of them against the oracle as well
    o = oracle.waveform_inputs(ws[2], nthreads=oracle_threads())
    if prec == F.FEW_FP64:
        assert rel_l2(first[2], o) <= FP64_REL_L2
    else:
        assert oracle.mismatch(first[2], o) <= MIXED_MISMATCH
    for tr in trs:
        tr.release()


def test_batch_without_graph_and_with_spline_rebuild(gpu_ctx):
    import torch
    ws = _mixed_set(11)[:4]
    trs = [RT.from_inputs(gpu_ctx, w) for w in ws]
    outs = [RT.alloc_out(w.n_samples, True) for w in ws]
    reqs = [RT.request(tr, o, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_MIXED, w.scale)
            for tr, o, w in zip(trs, outs, ws)]
    b1 = F.few_batch_plan(gpu_ctx.handle, reqs, F.FEW_BATCH_NO_GRAPH)
    b2 = F.few_batch_plan(gpu_ctx.handle, reqs, F.FEW_BATCH_REBUILD_SPLINES)
    F.few_batch_run(gpu_ctx.handle, b1, RT.current_stream())
    torch.cuda.synchronize()
    h1 = [to_host(o) for o in outs]
    # change the knot data in place on the device; the rebuilding batch must pick it up
    for tr in trs:
        for t in tr._dev_inputs[2:]:
            t.mul_(0.5)
    F.few_batch_run(gpu_ctx.handle, b2, RT.current_stream())
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    for o, h in zip(outs, h1):
        g = to_host(o)
        assert np.max(np.abs(g - 0.5 * h)) <= 1e-5 * np.max(np.abs(h))
    F.few_batch_release(gpu_ctx.handle, b1)
    F.few_batch_release(gpu_ctx.handle, b2)
    for tr in trs:
        tr.release()


def test_batch_rejects_mixed_precisions_and_host_outputs(gpu_ctx):
    ws = _mixed_set()[:2]
    trs = [RT.from_inputs(gpu_ctx, w) for w in ws]
    o0 = RT.alloc_out(ws[0].n_samples, False)
    o1 = RT.alloc_out(ws[1].n_samples, True)
    r0 = RT.request(trs[0], o0, ws[0].n_samples, 0.0, ws[0].dt, 0.1, 0.2, F.FEW_FP64)
    r1 = RT.request(trs[1], o1, ws[1].n_samples, 0.0, ws[1].dt, 0.1, 0.2, F.FEW_MIXED)
    with pytest.raises(F.FewError):
        F.few_batch_plan(gpu_ctx.handle, [r0, r1])
    host = np.zeros(ws[0].n_samples, dtype=np.complex128)
    rh = RT.request(trs[0], host, ws[0].n_samples, 0.0, ws[0].dt, 0.1, 0.2, F.FEW_FP64,
                    out_where=F.FEW_MEM_HOST)
    with pytest.raises(F.FewError):
        F.few_batch_plan(gpu_ctx.handle, [rh])
    for tr in trs:
        tr.release()


def test_batch_of_256_uneven_waveforms(gpu_ctx):
    """The 256-waveform batch workload in one persistent graph launch; oracle on windows."""
    import torch
    ws = W.config3(256)
    counts = [w.N for w in ws]
    assert min(counts) >= 10 and max(counts) <= 3843
    trs = [RT.from_inputs(gpu_ctx, w) for w in ws]
    outs = [RT.alloc_out(w.n_samples, True) for w in ws]
    reqs = [RT.request(tr, o, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_MIXED, w.scale)
            for tr, o, w in zip(trs, outs, ws)]
    b = F.few_batch_plan(gpu_ctx.handle, reqs, F.FEW_BATCH_REBUILD_SPLINES)
    F.few_batch_run(gpu_ctx.handle, b, RT.current_stream())
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    rng = np.random.default_rng(3)
    for q in rng.choice(len(ws), size=6, replace=False):
        w = ws[q]
        i0 = int(rng.integers(0, w.n_samples - 1500))
        o = oracle.waveform_inputs(w, i0, 1500, nthreads=oracle_threads())
        g = outs[q][i0:i0 + 1500].cpu().numpy()
        assert oracle.mismatch(g, o) <= MIXED_MISMATCH, (q, w.N)
    F.few_batch_release(gpu_ctx.handle, b)
    for tr in trs:
        tr.release()
