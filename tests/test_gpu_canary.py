"""Host-side canaries around output buffers.

Every output is a window of a larger device buffer whose guard regions hold a sentinel; after
the call the guards must be untouched and the window fully written.  The sample counts are
ragged against every tile (a pass of threads x R samples, warps of 32 x R, anchor groups of 16),
so a store past the last sample of a pass, of a segment or of the waveform would show.
"""
import numpy as np
import pytest

from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 4099  # elements on each side: odd, a multiple of no tile
SENTINEL = complex(1234.5, -987.25)


def _guarded(n, c64):
    import torch
    dt = torch.complex64 if c64 else torch.complex128
    buf = torch.full((n + 2 * GUARD,), SENTINEL, dtype=dt, device="cuda")
    return buf, buf[GUARD:GUARD + n]


def _check(buf, lo, n):
    h = buf.cpu().numpy()
    s = h.dtype.type(SENTINEL)
    assert np.all(h[:lo] == s) and np.all(h[lo + n:] == s), "a guard was overwritten"
    win = h[lo:lo + n]
    assert np.all(np.isfinite(win)) and not np.any(win == s), "the window was not fully written"


@pytest.mark.parametrize("ns", [1, 31, 1023, 1025, 4097, 60480])
@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
def test_waveform_writes_only_its_output(gpu_ctx, ns, prec):
    import torch
    w = W.config1()
    tr = RT.from_inputs(gpu_ctx, w)
    buf, out = _guarded(ns, prec == F.FEW_MIXED)
    req = RT.request(tr, out, ns, w.t0, w.dt, w.theta, w.phi, prec)
    F.few_waveform(gpu_ctx.handle, req, RT.current_stream())
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    tr.release()
    _check(buf, GUARD, ns)


@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
def test_batch_writes_only_its_outputs(gpu_ctx, prec):
    """Ragged waveforms of one batch write into windows of one buffer separated by guards."""
    import torch
    sizes = [1, 17, 255, 257, 2049, 5000]
    ws = [W.tiny_inputs(300 + k, K=5 + k, n_samples=max(n, 2)) for k, n in enumerate(sizes)]
    c64 = prec == F.FEW_MIXED
    total = sum(sizes) + GUARD * (len(sizes) + 1)
    dt = torch.complex64 if c64 else torch.complex128
    buf = torch.full((total,), SENTINEL, dtype=dt, device="cuda")
    trs, reqs, offs, pos = [], [], [], GUARD
    for w, n in zip(ws, sizes):
        tr = RT.from_inputs(gpu_ctx, w)
        trs.append(tr)
        reqs.append(RT.request(tr, buf[pos:pos + n], n, w.t0, w.dt, w.theta, w.phi, prec))
        offs.append(pos)
        pos += n + GUARD
    b = F.few_batch_plan(gpu_ctx.handle, reqs)
    F.few_batch_run(gpu_ctx.handle, b, RT.current_stream())
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    F.few_batch_release(gpu_ctx.handle, b)
    for tr in trs:
        tr.release()
    h = buf.cpu().numpy()
    s = h.dtype.type(SENTINEL)
    edges = [0] + [x for o, n in zip(offs, sizes) for x in (o, o + n)] + [total]
    for a, e in zip(edges[0::2], edges[1::2]):  # the guards between the windows
        assert np.all(h[a:e] == s), (a, e)
    for o, n in zip(offs, sizes):
        win = h[o:o + n]
        assert np.all(np.isfinite(win)) and not np.any(win == s)
