"""Serving loop on the GPU: an MCMC-like Poisson stream of requests (durations 0.5-4 yr, dt in
{5, 10, 15} s, 10-1000 modes, perturbed angles/phases/scale of resident trajectories).  Requests
that arrive while others run are admitted as memory frees up; each result must be the same
alone and in the mix (bit-identical), and the latency statistics must be populated.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W
from paper_2104_04582_gb300.serve import GpuEngine, Request, Server
from tests.gpu_common import MIXED_MISMATCH, oracle_threads, to_host

pytestmark = pytest.mark.gpu


def _requests(trajs, stream):
    out = []
    for r in stream:
        w = trajs[r.traj_key]
        out.append(Request(traj_key=r.traj_key, n_samples=w.n_samples, dt=w.dt, t0=w.t0,
                           theta=r.theta, phi=r.phi, scale=r.scale, dphi_phi0=r.dphi_phi0,
                           dphi_r0=r.dphi_r0, prec=F.FEW_MIXED))
    return out


@pytest.mark.parametrize("budget_gb", [64.0, 1.5])
def test_serving_results_same_alone_and_in_the_mix(gpu_ctx, budget_gb):
    import torch
    trajs_in, stream = W.config4_stream(24, rate_hz=400.0, seed=W.SEEDS["C4"] + int(budget_gb))
    trajs = {k: RT.from_inputs(gpu_ctx, w) for k, w in trajs_in.items()}
    reqs = _requests(trajs_in, stream)
    srv = Server(GpuEngine(gpu_ctx, trajs), hbm_budget_bytes=int(budget_gb * 2 ** 30),
                 max_batch=8, max_inflight=3)
    t0 = time.perf_counter()
    futs = []
    for r, s in zip(reqs, stream):
        delay = s.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        futs.append(srv.submit(r))
    assert srv.drain(timeout=600)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert np.isfinite(st["p50_ms"]) and st["p99_ms"] >= st["p50_ms"]
    assert st["max_bytes_in_use"] <= int(budget_gb * 2 ** 30)
    # same alone and in the mix
    for r, f in zip(reqs, futs):
        got = to_host(f.result())
        tr = trajs[r.traj_key]
        alone = RT.waveform(gpu_ctx, tr, r.n_samples, r.t0, r.dt, r.theta, r.phi, r.prec,
                            scale=r.scale, dphi_phi0=r.dphi_phi0, dphi_r0=r.dphi_r0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_host(alone), got)
    # and one of them against the oracle
    r = reqs[0]
    w = trajs_in[r.traj_key]
    o = oracle.waveform(w.t_knots, w.phi_phi + r.dphi_phi0, w.phi_r + r.dphi_r0, w.modes,
                        w.amp_re, w.amp_im, r.theta, r.phi, r.scale, r.t0, r.dt, 0, 2000,
                        oracle_threads())
    assert oracle.mismatch(to_host(futs[0].result())[:2000], o) <= MIXED_MISMATCH
    srv.close()
    for tr in trajs.values():
        tr.release()


def test_serving_creates_new_trajectories_on_first_use(gpu_ctx):
    """An engine that starts empty: the first request of each trajectory brings its knot data,
    the engine creates the trajectory and builds its splines on that request's path, later
    requests reuse it; the results equal those on trajectories created beforehand."""
    import torch
    trajs_in, stream = W.config4_stream(20, rate_hz=400.0, seed=W.SEEDS["C4"] + 7, p_new=0.3)
    reqs, seen = [], set()
    for r in _requests(trajs_in, stream):
        if r.traj_key not in seen:
            r.traj_inputs = trajs_in[r.traj_key]
            seen.add(r.traj_key)
        reqs.append(r)
    assert len(seen) >= 3
    engine = GpuEngine(gpu_ctx)
    srv = Server(engine, hbm_budget_bytes=8 * 2 ** 30, max_batch=4, max_inflight=2)
    futs = [srv.submit(r) for r in reqs]
    assert srv.drain(timeout=600)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert sorted(engine.trajs) == sorted(seen)
    ref = {k: RT.from_inputs(gpu_ctx, w) for k, w in trajs_in.items()}
    for r, f in zip(reqs, futs):
        alone = RT.waveform(gpu_ctx, ref[r.traj_key], r.n_samples, r.t0, r.dt, r.theta, r.phi,
                            r.prec, scale=r.scale, dphi_phi0=r.dphi_phi0, dphi_r0=r.dphi_r0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_host(alone), to_host(f.result()))
    srv.close()
    engine.close()
    assert not engine.trajs
    for tr in ref.values():
        tr.release()
