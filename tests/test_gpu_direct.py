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
