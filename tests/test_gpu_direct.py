"""Direct (non-interpolated) summation (Sec. 3.C) on the GPU against the oracle, with the
amplitudes and phases of the synthetic inspiral given at every sample."""
import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W
from tests.gpu_common import FP64_REL_L2, MIXED_MISMATCH, oracle_threads, rel_l2, to_host

pytestmark = pytest.mark.gpu


def _dense(w, ns, i0=0):
    ts = w.t0 + (i0 + np.arange(ns)) * w.dt
    pphi, pr = w.phases_at(ts)
    A = w.amp_model(ts)
    return pphi, pr, np.ascontiguousarray(A.real), np.ascontiguousarray(A.imag)


def _gpu_direct(ctx, pphi, pr, are, aim, modes, theta, phi, prec):
    import torch
    t = [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in (pphi, pr, are, aim)]
    out = torch.empty(len(pphi), dtype=torch.complex64 if prec == F.FEW_MIXED else torch.complex128,
                      device="cuda")
    F.few_direct_sum(ctx.handle, *t, modes, theta, phi, out, 1.0, prec, RT.current_stream())
    torch.cuda.synchronize()
    return to_host(out)


@pytest.mark.parametrize("cfg,ns,i0", [("week", 20000, 0), ("year", 2000, 3000000)])
@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
def test_direct_matches_oracle(gpu_ctx, cfg, ns, i0, prec):
    w = W.config1() if cfg == "week" else W.config2()
    pphi, pr, are, aim = _dense(w, ns, i0)
    g = _gpu_direct(gpu_ctx, pphi, pr, are, aim, w.modes, w.theta, w.phi, prec)
    o = oracle.direct_dense(pphi, pr, w.modes, are, aim, w.theta, w.phi, 1.0, oracle_threads())
    if prec == F.FEW_FP64:
        assert rel_l2(g, o) <= FP64_REL_L2
    else:
        assert oracle.mismatch(g, o) <= MIXED_MISMATCH


@pytest.mark.parametrize("N,ns", [(1, 1), (33, 777), (97, 5)])
def test_direct_ragged_sizes(gpu_ctx, N, ns):
    w = W.config1()
    idx = np.arange(N)
    modes = w.modes[idx]
    pphi, pr, are, aim = _dense(w, ns, 1234)
    g = _gpu_direct(gpu_ctx, pphi, pr, are[:, idx], aim[:, idx], modes, 0.7, 1.9, F.FEW_FP64)
    o = oracle.direct_dense(pphi, pr, modes, are[:, idx], aim[:, idx], 0.7, 1.9)
    assert rel_l2(g, o) <= FP64_REL_L2


def test_direct_mixed_amplitude_range(gpu_ctx):
    """The mixed path converts FP64 amplitudes to FP32 on the integer pipe (round to nearest,
    ties away from zero, magnitudes below 2^-126 flushed to zero).  One m = 0 mode at zero phase makes every output
    sample a single product A_i * -2Y_20, so each conversion branch (zero, below the normal
    range, boundary magnitudes, exact rounding ties, the whole normal range) is checked sample
    by sample against the oracle: within FP32 rounding, plus the flush's absolute 2^-126."""
    rng = np.random.default_rng(20240417)
    ns = 4096
    amp = (rng.standard_normal(ns) + 1j * rng.standard_normal(ns)) * 10.0 ** rng.uniform(-37, 37, ns)
    special = np.array([0.0, -0.0, 1e-39, -3e-42, 2.0 ** -126, -(2.0 ** -126) * (1 - 2.0 ** -30),
                        2.0 ** -149, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, -(1.0 + 2.0 ** -24),
                        3.0e38, -2.0 ** 127])
    amp[:len(special)] = special * (1 + 1j)           # both parts special, same sample
    amp[len(special):2 * len(special)] = special      # real part special, imaginary part zero
    are = np.ascontiguousarray(amp.real.reshape(ns, 1))
    aim = np.ascontiguousarray(amp.imag.reshape(ns, 1))
    modes = np.array([[2, 0, 0]], dtype=np.int32)
    zeros = np.zeros(ns)
    g = _gpu_direct(gpu_ctx, zeros, zeros, are, aim, modes, 0.7, 0.0, F.FEW_MIXED)
    o = oracle.direct_dense(zeros, zeros, modes, are, aim, 0.7, 0.0)
    err = np.abs(g.astype(np.complex128) - o)
    assert np.all(err <= 1e-6 * np.abs(o) + 2.0 ** -126), np.max(err / (np.abs(o) + 1e-300))
    assert np.all(g[o == 0] == 0)


@pytest.mark.parametrize("N,ns", [(64, 3), (97, 777), (513, 152), (3843, 301)])
def test_direct_mixed_sizes(gpu_ctx, N, ns):
    """Mixed path at mode counts from 64 to the full grid, sample counts below and above the
    number of warps in flight, and odd N (rows that start 8 bytes past a 16-byte boundary)."""
    w = W.config2()
    idx = np.arange(N)
    modes = w.modes[idx]
    pphi, pr, are, aim = _dense(w, ns, 2000000)
    are, aim = np.ascontiguousarray(are[:, idx]), np.ascontiguousarray(aim[:, idx])
    g = _gpu_direct(gpu_ctx, pphi, pr, are, aim, modes, w.theta, w.phi, F.FEW_MIXED)
    o = oracle.direct_dense(pphi, pr, modes, are, aim, w.theta, w.phi, 1.0, oracle_threads())
    assert oracle.mismatch(g, o) <= MIXED_MISMATCH


def test_direct_mixed_unaligned_amplitudes(gpu_ctx):
    """Amplitude arrays that start 8 bytes past a 16-byte boundary (a sliced view) give the
    oracle's result."""
    import torch
    w = W.config1()
    ns = 3001
    pphi, pr, are, aim = _dense(w, ns)
    N = are.shape[1]
    d = [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in (pphi, pr)]
    views = []
    for a in (are, aim):
        buf = torch.zeros(ns * N + 1, dtype=torch.float64, device="cuda")
        buf[1:] = torch.as_tensor(a.ravel()).cuda()
        views.append(buf[1:])
    assert views[0].data_ptr() % 16 == 8
    out = torch.empty(ns, dtype=torch.complex64, device="cuda")
    F.few_direct_sum(gpu_ctx.handle, d[0], d[1], views[0], views[1], w.modes, w.theta, w.phi, out,
                     1.0, F.FEW_MIXED, RT.current_stream())
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    o = oracle.direct_dense(pphi, pr, w.modes, are, aim, w.theta, w.phi, 1.0, oracle_threads())
    assert oracle.mismatch(to_host(out), o) <= MIXED_MISMATCH
