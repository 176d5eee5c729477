"""Host logic of the serving loop, on the CPU with a fake engine (no GPU).

Admission by memory budget (FIFO, head-of-line), batching by precision, overlap of several
groups in flight, cancellation, and host-side fault injection (refused admission, failed
allocation, a failing launch), plus the latency statistics.
"""
import threading
import time

import pytest

from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300.serve import AdmissionError, FaultInjector, Request, Server


class FakeEngine:
    """Runs each group on a timer thread; the result is the tuple of request parameters."""

    def __init__(self, seconds_per_sample=2e-7, fail_launch=lambda reqs: False):
        self.sps = seconds_per_sample
        self.fail_launch = fail_launch
        self.groups = []
        self.active = 0
        self.max_active = 0
        self.lock = threading.Lock()

    def scratch_bytes(self, req):
        return 1000

    def alloc_out(self, req):
        return {"req": req}

    def launch(self, reqs, outs):
        if self.fail_launch(reqs):
            raise RuntimeError("launch failed (injected)")
        self.groups.append([r.traj_key for r in reqs])
        done = threading.Event()
        dur = self.sps * sum(r.n_samples for r in reqs)
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)

        def run():
            time.sleep(dur)
            for o in outs:
                o["value"] = (o["req"].traj_key, o["req"].theta)
            with self.lock:
                self.active -= 1
            done.set()
        threading.Thread(target=run, daemon=True).start()
        return done

    def wait(self, handle):
        handle.wait(10)

    def release(self, handle):
        pass


def _req(k, n=10000, prec=F.FEW_MIXED):
    return Request(traj_key=k, n_samples=n, dt=10.0, theta=0.1 * k, prec=prec)


def test_all_requests_complete_with_results_in_order():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget_bytes=10 ** 9, max_batch=4, max_inflight=3)
    futs = [srv.submit(_req(k)) for k in range(25)]
    assert srv.drain(timeout=20)
    for k, f in enumerate(futs):
        assert f.result()["value"] == (k, 0.1 * k)
    st = srv.stats()
    assert st["completed"] == 25 and st["failed"] == 0
    assert st["p50_ms"] <= st["p99_ms"]
    assert max(len(g) for g in eng.groups) <= 4
    srv.close()


def test_budget_limits_memory_in_flight():
    eng = FakeEngine(seconds_per_sample=1e-6)
    per = 10000 * 8 + 1000
    srv = Server(eng, hbm_budget_bytes=2 * per + 10, max_batch=8, max_inflight=8)
    futs = [srv.submit(_req(k)) for k in range(10)]
    assert srv.drain(timeout=30)
    assert all(f.done() and not f.exception() for f in futs)
    assert srv.stats()["max_bytes_in_use"] <= 2 * per + 10
    srv.close()


def test_oversized_request_is_refused_immediately():
    srv = Server(FakeEngine(), hbm_budget_bytes=50000)
    f = srv.submit(_req(1, n=10 ** 6))
    with pytest.raises(AdmissionError):
        f.result(timeout=1)
    srv.close()


def test_groups_keep_one_precision():
    eng = FakeEngine()
    srv = Server(eng, hbm_budget_bytes=10 ** 9, max_batch=16, max_inflight=1)
    futs = [srv.submit(_req(k, prec=F.FEW_FP64 if k % 3 == 0 else F.FEW_MIXED)) for k in range(12)]
    assert srv.drain(timeout=20)
    for g in eng.groups:
        precs = {F.FEW_FP64 if k % 3 == 0 else F.FEW_MIXED for k in g}
        assert len(precs) == 1
    assert all(not f.exception() for f in futs)
    srv.close()


def test_overlap_of_groups_in_flight():
    eng = FakeEngine(seconds_per_sample=5e-6)
    srv = Server(eng, hbm_budget_bytes=10 ** 9, max_batch=1, max_inflight=3)
    for k in range(9):
        srv.submit(_req(k))
    assert srv.drain(timeout=30)
    assert eng.max_active >= 2
    assert srv.stats()["max_inflight_batches"] <= 3
    srv.close()


def test_fault_injection_and_cancellation():
    faults = FaultInjector(reject_admission=lambda r: r.traj_key == 3,
                           fail_allocation=lambda r: r.traj_key == 5)
    eng = FakeEngine(seconds_per_sample=2e-6, fail_launch=lambda reqs: any(r.traj_key == 7 for r in reqs))
    srv = Server(eng, hbm_budget_bytes=10 ** 9, max_batch=1, max_inflight=1, faults=faults)
    futs = [srv.submit(_req(k)) for k in range(10)]
    cancelled = futs[9].cancel()  # still queued behind the others
    assert srv.drain(timeout=30)
    with pytest.raises(AdmissionError):
        futs[3].result()
    with pytest.raises(MemoryError):
        futs[5].result()
    with pytest.raises(RuntimeError):
        futs[7].result()
    if cancelled:
        assert futs[9].cancelled()
    for k in (0, 1, 2, 4, 6, 8):
        assert futs[k].result()["value"][0] == k
    st = srv.stats()
    assert st["failed"] == 3
    srv.close()


def test_request_that_cannot_be_sized_is_refused_through_its_future():
    """An engine that cannot size a request (an unknown trajectory without knot data) refuses
    it through the future; the server keeps serving the others."""
    class Picky(FakeEngine):
        def scratch_bytes(self, req):
            if req.traj_key == 2:
                raise KeyError("unknown trajectory 2 and no knot data")
            return 1000
    eng = Picky()
    srv = Server(eng, hbm_budget_bytes=10 ** 9, max_batch=4, max_inflight=2)
    futs = [srv.submit(_req(k)) for k in range(5)]
    assert srv.drain(timeout=20)
    with pytest.raises(AdmissionError, match="cannot be sized"):
        futs[2].result()
    assert [futs[k].result()["value"][0] for k in (0, 1, 3, 4)] == [0, 1, 3, 4]
    srv.close()
