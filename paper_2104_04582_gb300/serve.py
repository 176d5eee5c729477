"""Serving loop: continuous batching of waveform requests with HBM-budget admission.

Requests arrive as an MCMC sampler emits them (different durations, cadences, mode counts,
angles and phase offsets of resident trajectories).  The server

* keeps trajectory splines resident on the device (registered once per trajectory key); a
  request may bring the knot data of a trajectory the server does not hold yet, which is then
  created and its splines built on that request's path (the paper's sampler proposes new
  trajectories as well as new angles and phases of known ones);
* admits queued requests in arrival order while their device memory (output + plan scratch)
  fits the HBM budget and a launch slot is free -- requests that arrive while others run are
  admitted as soon as slots and memory free up;
* launches each admitted group as one batched persistent summation (one plan, one launch
  sequence) on one of several worker streams, so the work of successive groups overlaps on the
  device;
* resolves each request's Future when its group's completion event fires, releases its memory
  and records submit-to-result latency (p50/p99) and throughput.

Each result is bit-identical to the same request run alone: every sample is summed by one thread
in an order fixed by the request's own mode table, whatever else shares the launch.

The execution engine is pluggable: `GpuEngine` drives libfewsum.so; tests of the host logic
(admission, batching, faults) use a fake engine on the CPU.  Fault injection is host-side only
(`FaultInjector`): forced admission rejection, forced allocation failure, and cancellation.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Any, Callable, Deque, Dict, List, Optional

from . import fewsum as F
from . import tune


class AdmissionError(RuntimeError):
    """The request can never fit the budget, or admission was refused."""


@dataclasses.dataclass
class Request:
    traj_key: Any
    n_samples: int
    dt: float
    t0: float = 0.0
    theta: float = 0.0
    phi: float = 0.0
    scale: float = 1.0
    dphi_phi0: float = 0.0
    dphi_r0: float = 0.0
    prec: int = F.FEW_MIXED
    out_c64: Optional[bool] = None
    # knot data (t_knots, modes, phi_phi, phi_r, amp_re, amp_im) of a trajectory the engine may
    # not hold yet: created under traj_key before the first group that uses it runs
    traj_inputs: Any = None

    def c64(self) -> bool:
        return self.prec == F.FEW_MIXED if self.out_c64 is None else bool(self.out_c64)

    def out_bytes(self) -> int:
        return self.n_samples * (8 if self.c64() else 16)


@dataclasses.dataclass
class FaultInjector:
    """Host-side faults for tests: each hook gets the request and returns True to fire."""
    reject_admission: Callable[[Request], bool] = lambda r: False
    fail_allocation: Callable[[Request], bool] = lambda r: False


@dataclasses.dataclass
class _Job:
    req: Request
    fut: cf.Future
    t_submit: float
    need: int = 0
    out: Any = None


class Server:
    def __init__(self, engine, hbm_budget_bytes: int, max_batch: int = 32, max_inflight: int = 3,
                 faults: Optional[FaultInjector] = None):
        self.engine = engine
        self.budget = int(hbm_budget_bytes)
        self.max_batch = int(max_batch)
        self.max_inflight = int(max_inflight)
        self.faults = faults or FaultInjector()
        self._q: Deque[_Job] = collections.deque()
        self._inflight: Deque[tuple] = collections.deque()  # (handle, [jobs], bytes)
        self._in_use = 0
        self._pending = 0  # submitted jobs whose future is not settled yet
        self._cv = threading.Condition()
        self._stop = False
        self.latencies: List[float] = []
        self.completed = 0
        self.failed = 0
        self.max_seen_inflight = 0
        self.max_seen_bytes = 0
        self.t_first = None
        self.t_last = None
        self._sched = threading.Thread(target=self._schedule_loop, name="fewsum-sched", daemon=True)
        self._done = threading.Thread(target=self._complete_loop, name="fewsum-done", daemon=True)
        self._sched.start()
        self._done.start()

    # ------------------------------------------------------------------ API
    def submit(self, req: Request) -> cf.Future:
        fut: cf.Future = cf.Future()
        try:
            need = req.out_bytes() + self.engine.scratch_bytes(req)
        except Exception as e:  # noqa: BLE001 -- e.g. an unknown trajectory without knot data
            fut.set_exception(AdmissionError(f"request cannot be sized: {e}"))
            return fut
        if need > self.budget:
            fut.set_exception(AdmissionError(f"request needs {need} bytes > budget {self.budget}"))
            return fut
        job = _Job(req, fut, time.perf_counter(), need)
        with self._cv:
            if self._stop:
                raise RuntimeError("server closed")
            self._q.append(job)
            self._pending += 1
            self._cv.notify_all()
        return fut

    def drain(self, timeout: Optional[float] = None) -> bool:
        """Wait until the queue is empty and nothing is in flight."""
        t_end = None if timeout is None else time.perf_counter() + timeout
        with self._cv:
            while self._pending > 0:
                rem = None if t_end is None else t_end - time.perf_counter()
                if rem is not None and rem <= 0:
                    return False
                self._cv.wait(0.05 if rem is None else min(rem, 0.05))
        return True

    def close(self) -> None:
        self.drain()
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._sched.join()
        self._done.join()

    def stats(self) -> Dict[str, float]:
        lat = sorted(self.latencies)

        def pct(p):
            if not lat:
                return float("nan")
            k = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
            return lat[k]
        span = (self.t_last - self.t_first) if (self.t_first and self.t_last) else float("nan")
        return {"completed": self.completed, "failed": self.failed,
                "p50_ms": 1e3 * pct(50), "p99_ms": 1e3 * pct(99),
                "mean_ms": 1e3 * (sum(lat) / len(lat)) if lat else float("nan"),
                "waveforms_per_s": self.completed / span if span and span > 0 else float("nan"),
                "max_inflight_batches": self.max_seen_inflight,
                "max_bytes_in_use": self.max_seen_bytes}

    # ------------------------------------------------------------------ internals
    def _admit(self) -> List[_Job]:
        """Pop the longest FIFO prefix (same precision) that fits memory and the batch size."""
        group: List[_Job] = []
        while self._q and len(group) < self.max_batch:
            job = self._q[0]
            if job.fut.cancelled():
                self._q.popleft()
                self._pending -= 1
                self._cv.notify_all()
                continue
            if group and job.req.prec != group[0].req.prec:
                break
            if self._in_use + job.need > self.budget:
                break  # head of line waits for memory
            self._q.popleft()
            if self.faults.reject_admission(job.req):
                self.failed += 1
                self._pending -= 1
                job.fut.set_exception(AdmissionError("admission refused"))
                self._cv.notify_all()
                continue
            if not job.fut.set_running_or_notify_cancel():
                self._pending -= 1
                self._cv.notify_all()
                continue
            self._in_use += job.need
            group.append(job)
        self.max_seen_bytes = max(self.max_seen_bytes, self._in_use)
        return group

    def _schedule_loop(self) -> None:
        while True:
            with self._cv:
                while not self._stop and (not self._q or len(self._inflight) >= self.max_inflight):
                    self._cv.wait(0.05)
                if self._stop and not self._q:
                    return
                group = self._admit()
            if not group:
                with self._cv:
                    self._cv.wait(0.001)
                continue
            ok: List[_Job] = []
            for job in group:
                try:
                    if self.faults.fail_allocation(job.req):
                        raise MemoryError("allocation failed (injected)")
                    job.out = self.engine.alloc_out(job.req)
                    ok.append(job)
                except Exception as e:  # noqa: BLE001 -- reported through the future
                    self._finish(job, error=e)
            if not ok:
                continue
            try:
                handle = self.engine.launch([j.req for j in ok], [j.out for j in ok])
            except Exception as e:  # noqa: BLE001
                for job in ok:
                    self._finish(job, error=e)
                continue
            with self._cv:
                if self.t_first is None:
                    self.t_first = min(j.t_submit for j in ok)
                self._inflight.append((handle, ok))
                self.max_seen_inflight = max(self.max_seen_inflight, len(self._inflight))
                self._cv.notify_all()

    def _complete_loop(self) -> None:
        while True:
            with self._cv:
                while not self._inflight and not (self._stop and not self._q):
                    self._cv.wait(0.05)
                if not self._inflight:
                    if self._stop and not self._q:
                        return
                    continue
                handle, jobs = self._inflight[0]
            err = None
            try:
                self.engine.wait(handle)
            except Exception as e:  # noqa: BLE001
                err = e
            self.engine.release(handle)
            now = time.perf_counter()
            with self._cv:
                self._inflight.popleft()
                for job in jobs:
                    self._finish_locked(job, now, err)
                self.t_last = now
                self._cv.notify_all()

    def _finish(self, job: _Job, error=None) -> None:
        with self._cv:
            self._finish_locked(job, time.perf_counter(), error)
            self._cv.notify_all()

    def _finish_locked(self, job: _Job, now: float, error) -> None:
        self._in_use -= job.need
        self._pending -= 1
        if error is not None:
            self.failed += 1
            if not job.fut.done():
                job.fut.set_exception(error)
            return
        self.completed += 1
        self.latencies.append(now - job.t_submit)
        if not job.fut.done():
            job.fut.set_result(job.out)


class GpuEngine:
    """Executes request groups with libfewsum.so: one batched plan per group, worker streams."""

    def __init__(self, ctx, trajectories: Optional[Dict[Any, Any]] = None, n_streams: int = 3):
        import torch
        self.torch = torch
        self.ctx = ctx
        # key -> runtime.Trajectory (spline data set); the caller's stay the caller's
        self.trajs: Dict[Any, Any] = dict(trajectories or {})
        self._owned: List[Any] = []  # keys of trajectories this engine created
        self._ready: Dict[Any, Any] = {}  # key -> event after its spline build
        # knot data announced by submitted requests, until their trajectory exists (later
        # requests of a new trajectory may be submitted before the first one runs)
        self._announced: Dict[Any, Any] = {}
        self.streams = [torch.cuda.Stream(device=ctx.device) for _ in range(n_streams)]
        self._next = 0
        self.tiles: Dict[int, tuple] = {}  # precision -> installed (R, threads, stage_slots)

    def _ensure_traj(self, req: Request, stream) -> Any:
        """The request's trajectory, created from its knot data (splines built on `stream`)
        if the engine does not hold it yet."""
        tr = self.trajs.get(req.traj_key)
        if tr is None:
            w = req.traj_inputs if req.traj_inputs is not None else self._announced.get(req.traj_key)
            if w is None:
                raise KeyError(f"unknown trajectory {req.traj_key!r} and no knot data")
            from . import runtime as RT
            tr = RT.Trajectory(self.ctx, w.t_knots, w.modes)
            try:
                tr.set_data_host(w.phi_phi, w.phi_r, w.amp_re, w.amp_im,
                                 stream=int(stream.cuda_stream))
            except Exception:
                tr.release()
                raise
            ev = self.torch.cuda.Event()
            ev.record(stream)  # groups on other streams wait for the build
            self.trajs[req.traj_key] = tr
            self._ready[req.traj_key] = ev
            self._owned.append(req.traj_key)
            self._announced.pop(req.traj_key, None)
        return tr

    def close(self) -> None:
        """Release the trajectories this engine created (their work must have completed)."""
        for k in self._owned:
            tr = self.trajs.pop(k, None)
            self._ready.pop(k, None)
            if tr is not None:
                tr.release()
        self._owned = []
        self._announced.clear()

    def tune_tiles(self, req: Request, cache_path: Optional[str] = tune.DEFAULT_CACHE) -> tuple:
        """Install the tile of `req`'s workload bucket (tuning on a cache miss, timed on `req`
        itself) for its precision; every later group of that precision runs with it."""
        torch = self.torch
        tr = self._ensure_traj(req, self.streams[0])
        torch.cuda.synchronize()
        K, N, slots = tr.info
        out = self.alloc_out(req)
        rq = F.make_request(tr.handle, out.data_ptr(), req.n_samples, req.t0, req.dt, req.theta,
                            req.phi, req.scale, req.prec, req.c64(), F.FEW_MEM_DEVICE,
                            req.dphi_phi0, req.dphi_r0)
        run = lambda: F.few_waveform(self.ctx.handle, rq, int(torch.cuda.current_stream().cuda_stream))
        choice, _ = tune.ensure(self.ctx.handle, run, req.prec, slots, req.n_samples, cache_path)
        torch.cuda.synchronize()
        self.tiles[req.prec] = tuple(choice)
        return tuple(choice)

    def scratch_bytes(self, req: Request) -> int:
        """Plan scratch of `req` (called by Server.submit for every request, which also lets
        the engine note the knot data a request brings)."""
        tr = self.trajs.get(req.traj_key)
        if req.traj_inputs is not None and tr is None:
            self._announced.setdefault(req.traj_key, req.traj_inputs)
        if tr is not None:
            K, N, slots = tr.info
        else:  # not created yet: sized from its knot data
            w = self._announced.get(req.traj_key)
            if w is None:
                raise KeyError(f"unknown trajectory {req.traj_key!r} and no knot data")
            K, slots = len(w.t_knots), F.few_mode_slots(w.modes)[0]
        elem = 8 if req.prec == F.FEW_FP64 else 4
        return (K - 1) * slots * 8 * elem + 64 * 1024

    def alloc_out(self, req: Request):
        torch = self.torch
        dt = torch.complex64 if req.c64() else torch.complex128
        s = self.streams[self._next % len(self.streams)]
        with torch.cuda.stream(s):
            return torch.empty(req.n_samples, dtype=dt, device=torch.device("cuda", self.ctx.device))

    def launch(self, reqs: List[Request], outs: List[Any]):
        torch = self.torch
        s = self.streams[self._next % len(self.streams)]
        self._next += 1
        for r in reqs:
            self._ensure_traj(r, s)
        for k in {r.traj_key for r in reqs}:
            ev = self._ready.get(k)
            if ev is not None:
                s.wait_event(ev)
        rq = [F.make_request(self.trajs[r.traj_key].handle, o.data_ptr(), r.n_samples, r.t0, r.dt,
                             r.theta, r.phi, r.scale, r.prec, r.c64(), F.FEW_MEM_DEVICE,
                             r.dphi_phi0, r.dphi_r0) for r, o in zip(reqs, outs)]
        b = F.few_batch_plan(self.ctx.handle, rq, F.FEW_BATCH_NO_GRAPH)
        F.few_batch_run(self.ctx.handle, b, int(s.cuda_stream))
        ev = torch.cuda.Event()
        ev.record(s)
        return (b, ev)

    def wait(self, handle) -> None:
        b, ev = handle
        ev.synchronize()

    def release(self, handle) -> None:
        b, ev = handle
        F.few_batch_release(self.ctx.handle, b)
