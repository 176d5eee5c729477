#!/usr/bin/env python3
"""Benchmark of the interpolated EMRI mode summation on GB300.

Workload (the configuration the headline metric is quoted on): one 1-yr waveform at dt = 10 s
(3,155,760 samples), K = 100 knots, the full 3843-mode Schwarzschild grid (l = 2..10,
m = 0..l, n = -30..30), synthetic seeded inputs.  A step is one pass of the whole hot path
with the knot data resident in HBM: spline build (all 7688 splines), harmonics, fold and the
per-sample mode sum, written to a device buffer.

Default arm (--impl gb300): the mixed-precision path (the fast path); the plain FP64 GPU path
is measured beside it.  Reference arm (--impl reference): the FP64 CPU oracle on the host cores,
on a bounded sample of the same workload, same metric.

One JSON line on stdout (rank 0).  Multi-GPU (torchrun): every rank computes its own
waveforms (independent problems, weak scaling, no collective on the data path); value is the
sum over ranks, timing the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2104_04582_gb300 import workloads as W  # noqa: E402

METRIC = "1-yr waveforms/s (3843 modes, dt=10 s) at mismatch<=1e-6; mode-samples/s vs plain FP64 path"
UNIT = "waveforms/s"
WORKLOAD = ("1-yr waveform, dt=10 s (3,155,760 samples), K=100 knots, 3843 modes "
            "(l=2..10, m=0..l, n=-30..30), m<0 by symmetry")
# DRAM bytes (read + write) of one summation launch on this workload, from the ncu capture
# summarised in profiles/k_sum_mixed_1yr_3843modes.md; used only while the kernel source is the
# one that was profiled (hash of sum.cu + phase_eval.cuh + async.cuh) and the tile is the
# profiled one.
PROFILED_TRAFFIC = {"source_sha256_16": "ea83547a100f196d", "tile": (4, 256), "bytes": 4113920 + 256}
N_SMS = 152
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25


def _kernel_source_hash() -> str:
    import hashlib
    d = os.path.join(ROOT, "paper_2104_04582_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("sum.cu", "phase_eval.cuh", "async.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks_file():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh)
    return {}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "sm_mhz_min": min(sm), "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU baseline (oracle)

def cpu_baseline(w, target_s: float = 12.0, max_samples=None):
    """The oracle, as it stands, on a bounded prefix of the workload, all host cores.

    A call costs a fixed part (all splines and harmonics) plus a part per sample; two short calls
    fit both, a third call of about `target_s` measures the per-sample rate, and the whole
    waveform's time is extrapolated as fixed + rate x N_s.
    """
    import oracle
    threads = os.cpu_count() or 1

    def run(n):
        t0 = time.perf_counter()
        h = oracle.waveform_inputs(w, 0, n, nthreads=threads)
        return time.perf_counter() - t0, h

    n1, n2 = 256, 2048
    t1, _ = run(n1)
    t2, _ = run(n2)
    per = max((t2 - t1) / (n2 - n1), 1e-12)
    fixed = max(t1 - per * n1, 0.0)
    n = int(min(w.n_samples, max(n2, (target_s - fixed) / per)))
    if max_samples:
        n = min(n, max_samples)
    el, h = run(n)
    per = max((el - fixed) / n, 1e-12)
    t_full = fixed + per * w.n_samples
    return {"value": 1.0 / t_full, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {n} of {w.n_samples} samples of the 1-yr 3843-mode waveform "
                      f"({n * w.N:.3g} mode-samples) in {el:.1f} s on {threads} OpenMP threads; "
                      f"fixed cost {fixed:.2f} s + {per * 1e6:.1f} us/sample extrapolated to the "
                      f"whole waveform ({t_full:.0f} s)",
            "mode_samples_per_s": n * w.N / max(el - fixed, 1e-9), "seconds": el,
            "seconds_full_waveform": t_full}, h


# ------------------------------------------------------------------ GPU arm

def _mismatch(a, b) -> float:
    """1 - overlap with unit noise (time-domain form), as 0.5*||a/|a| - b/|b|||^2."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    d = a / np.linalg.norm(a) - b / np.linalg.norm(b)
    return float(0.5 * np.vdot(d, d).real)


def l2_flush_buffer(torch, dev):
    return torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)


def _rb_device_inputs(M, N, n_traj, dev):
    import torch
    alpha, basis, nu = W.rb_inputs(M, 99, N, n_traj=n_traj)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    return (t(alpha.real), t(alpha.imag)), (t(basis.real), t(basis.imag)), t(nu)


def bench_rb(ctx, M, N, stream, sh):
    """Reduced-basis amplitudes for M knots (64 trajectories' worth by default), mixed precision
    with renormalisation, timed over the whole call; FP64 timed on one trajectory's knots."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    dev = torch.device("cuda", torch.cuda.current_device())
    (are, aim), (bre, bim), nu = _rb_device_inputs(M, N, max(1, M // 100), dev)
    Nb = int(are.shape[1])
    h = F.few_basis_create(ctx.handle, bre, bim, sh)
    ore = torch.empty((M, N), dtype=torch.float64, device=dev)
    oim = torch.empty_like(ore)

    def timed(m, prec, reps):
        F.few_rb_amplitudes(ctx.handle, h, are[:m], aim[:m], ore[:m], oim[:m], nu[:m], prec, sh)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for a, b_ in evs:
            a.record(stream)
            F.few_rb_amplitudes(ctx.handle, h, are[:m], aim[:m], ore[:m], oim[:m], nu[:m], prec, sh)
            b_.record(stream)
        torch.cuda.synchronize()
        return min(a.elapsed_time(b_) for a, b_ in evs)

    ms = timed(M, F.FEW_MIXED, 5)
    m64 = min(M, 100)
    ms64 = timed(m64, F.FEW_FP64, 3)
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("reduced-basis amplitudes latched an error")
    F.few_basis_release(ctx.handle, h)
    peaks = _peaks_file()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    nbytes = 16 * M * N + 16 * M * Nb + 16 * Nb * N + 8 * M  # out, alpha, basis, norms
    gbs = nbytes / (ms * 1e-3) / 1e9
    alg_flops = 8.0 * M * Nb * N  # complex product: 4 real multiply-adds per term
    n_kb = -(-(6 * Nb) // 64)  # three split products of depth 2 Nb
    # transposed tiles: 256 knots x 128 output columns (64 modes, real and imaginary)
    exec_flops = 2.0 * (-(-M // 256) * 256) * (-(-N // 64) * 128) * (n_kb * 64)
    return {"knots": M, "basis": Nb, "modes": N, "prec": "mixed (split fp16 on tcgen05)",
            "ms": ms, "amplitudes_per_s": M * N / (ms * 1e-3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "bytes_per_launch": nbytes,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"},
            "tensor": {"algorithmic_tflops": alg_flops / (ms * 1e-3) / 1e12,
                       "executed_tflops": exec_flops / (ms * 1e-3) / 1e12,
                       "executed_flops_per_launch": exec_flops, "peak": bf16,
                       "frac_executed": exec_flops / (ms * 1e-3) / 1e12 / bf16,
                       "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)"},
            "fp64": {"knots": m64, "ms": ms64}}


def measure_peaks(dev_index: int):
    """FP32 FMA, FP64 FMA and SFU rates from the probe library (ops/s, FMA = 1 op)."""
    import ctypes
    from paper_2104_04582_gb300 import _build
    if not os.path.exists(_build.PROBE_LIB):
        return {}
    L = ctypes.CDLL(_build.PROBE_LIB)
    L.fewprobe_measure.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]
    out = {}
    for which, name, it0 in ((0, "fp32_fma_per_s", 20000), (1, "fp64_fma_per_s", 400),
                             (2, "sfu_sin_per_s", 4000), (3, "fp32_fma_3reg_per_s", 20000),
                             (4, "fp32x2_fma_3reg_per_s", 10000),
                             (5, "fp32_fma_shared_addend_per_s", 20000),
                             (6, "fp32_fma_summation_block_per_s", 4000)):
        r, ms = ctypes.c_double(), ctypes.c_float()
        if L.fewprobe_measure(dev_index, which, it0, ctypes.byref(r), ctypes.byref(ms)):
            continue
        iters = int(it0 * max(1.0, 60.0 / max(ms.value, 1e-3)))
        if L.fewprobe_measure(dev_index, which, iters, ctypes.byref(r), ctypes.byref(ms)):
            continue
        out[name] = r.value
    return out


def dist_max(value: float, device=None) -> float:
    """Max of a per-rank float over the process group (any backend); identity when alone."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(ms_max: float, world: int, waveforms_per_rank_step: int = 1) -> float:
    """Whole-job waveforms/s: every rank computes its own waveforms each step (weak scaling)."""
    return world * waveforms_per_rank_step * 1000.0 / ms_max


def run_gpu(args, rank: int, world: int, local_rank: int):
    import torch
    from paper_2104_04582_gb300 import _build
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT

    _build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = W.config2(W.SEEDS["C2"] + rank)
    ctx = RT.Context(local_rank)
    F.few_ctx_set_timing(ctx.handle, True)
    stream = torch.cuda.current_stream(dev)
    sh = int(stream.cuda_stream)
    prec = F.FEW_MIXED if args.prec == "mixed" else F.FEW_FP64
    c64 = prec == F.FEW_MIXED

    tr = RT.Trajectory(ctx, w.t_knots, w.modes)
    dev_in = tr.upload_inputs(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
    tile = tuple(ctx.get_tiles(prec))
    out = RT.alloc_out(w.n_samples, c64, local_rank)
    req = RT.request(tr, out, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec)
    flush = l2_flush_buffer(torch, dev)
    K_, N_, slots = tr.info

    def step():
        F.few_traj_set_data(ctx.handle, tr.handle, *dev_in, stream=sh)
        F.few_waveform(ctx.handle, req, sh)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("device error during warm-up")

    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sum_ms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    F.few_ctx_set_timing(ctx.handle, False)  # the library's per-kernel events stay out of the timed steps
    for k in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (outside the step's events)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    F.few_ctx_set_timing(ctx.handle, True)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # the summation kernel's own duration (CUDA events the library records around it on the
    # same stream), read after each of a few more flushed steps; reading waits for the step, so
    # this runs after the timed loop rather than inside it
    for k in range(min(args.steps, 5)):
        flush.zero_()
        step()
        kt = F.few_last_timing(ctx.handle)
        sum_ms.append(kt[3])
    ms_local = sum(step_ms) / len(step_ms)
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("device error during the timed region")
    h_fast = out.cpu().numpy().astype(np.complex128) if rank == 0 else None
    kernel_ms = [float(x) for x in sum_ms if x > 0]
    last_t = F.few_last_timing(ctx.handle)

    # plain FP64 path on the same inputs (fewer steps: it is ~50x slower)
    plain = None
    h_plain = None
    if rank == 0 and not args.no_plain and prec == F.FEW_MIXED:
        out64 = RT.alloc_out(w.n_samples, False, local_rank)
        req64 = RT.request(tr, out64, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_FP64)
        F.few_traj_set_data(ctx.handle, tr.handle, *dev_in, stream=sh)
        F.few_waveform(ctx.handle, req64, sh)
        torch.cuda.synchronize()
        pk = max(2, min(5, args.steps))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(pk)]
        sum64 = []
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            F.few_traj_set_data(ctx.handle, tr.handle, *dev_in, stream=sh)
            F.few_waveform(ctx.handle, req64, sh)
            b.record(stream)
            sum64.append(F.few_last_timing(ctx.handle)[3])
        torch.cuda.synchronize()
        ms64 = sum(a.elapsed_time(b) for a, b in ev) / pk
        h_plain = out64.cpu().numpy()
        plain = {"ms_per_step": ms64, "value": 1000.0 / ms64, "unit": UNIT,
                 "mode_samples_per_s": w.N * w.n_samples / (ms64 * 1e-3),
                 "sum_kernel_ms": sum(sum64) / len(sum64), "dtype": "f64"}
        del out64

    # e2e through the C ABI with host buffers (pinned), copies inside the timed region
    F.few_ctx_set_timing(ctx.handle, False)  # no per-kernel events in the remaining timed loops
    e2e = None
    if rank == 0:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        h_in = [pin(a) for a in (w.phi_phi, w.phi_r, w.amp_re, w.amp_im)]
        host_out = torch.empty(w.n_samples, dtype=torch.complex64 if c64 else torch.complex128
                               ).pin_memory().numpy()
        req_h = RT.request(tr, host_out, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec,
                           out_where=F.FEW_MEM_HOST)
        e_steps = max(3, min(args.steps, 10))
        for _ in range(2):
            F.few_traj_set_data(ctx.handle, tr.handle, *h_in, stream=sh)
            F.few_waveform(ctx.handle, req_h, sh)
        torch.cuda.synchronize()
        t_e = []
        for _ in range(e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            F.few_traj_set_data(ctx.handle, tr.handle, *h_in, stream=sh)
            F.few_waveform(ctx.handle, req_h, sh)  # host output: returns after the D2H copy
            t_e.append(time.perf_counter() - t0)
        h2d = sum(a.nbytes for a in h_in)
        d2h = host_out.nbytes
        e2e = {"value": 1.0 / statistics.mean(t_e), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1000.0 * statistics.mean(t_e), "steps": e_steps,
               "timer": "host wall clock around the two C-ABI calls (the call with host output "
                        "returns once the result is in host memory; page-locked output is "
                        "stored by the summation kernel directly)"}

    # batched path: B independent 1-yr 3843-mode waveforms (own trajectories) per step, one
    # persistent summation launch, the whole sequence (spline rebuild included) as a CUDA graph
    batched = None
    if rank == 0 and args.batch > 1:
        wb = [W.config2(W.SEEDS["C2"] + 1000 + q) for q in range(args.batch)]
        trb = [RT.from_inputs(ctx, x) for x in wb]
        outb = [RT.alloc_out(x.n_samples, c64, local_rank) for x in wb]
        reqb = [RT.request(t_, o_, x.n_samples, x.t0, x.dt, x.theta, x.phi, prec)
                for t_, o_, x in zip(trb, outb, wb)]
        bh = F.few_batch_plan(ctx.handle, reqb, F.FEW_BATCH_REBUILD_SPLINES)
        for _ in range(2):
            F.few_batch_run(ctx.handle, bh, sh)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(max(3, min(args.steps, 10)))]
        for a, b_ in evs:
            flush.zero_()
            a.record(stream)
            F.few_batch_run(ctx.handle, bh, sh)
            b_.record(stream)
        torch.cuda.synchronize()
        if ctx.sync_status() != F.FEW_OK:
            raise RuntimeError("device error in the batched run")
        msb = sum(a.elapsed_time(b_) for a, b_ in evs) / len(evs)
        batched = {"waveforms_per_step": args.batch, "ms_per_step": msb,
                   "value": args.batch * 1000.0 / msb, "unit": UNIT,
                   "mode_samples_per_s": args.batch * w.N * w.n_samples / (msb * 1e-3),
                   "launches_per_step": 4, "graph": True,
                   "step": "spline rebuild of all trajectories + harmonics + fold + one "
                           "persistent summation launch, replayed as one CUDA graph"}
        F.few_batch_release(ctx.handle, bh)
        for t_ in trb:
            t_.release()
        del outb

    # Mode Selector (Sec. 3.D) on the benchmark's knot amplitudes, eps = 1e-5
    selector = None
    if rank == 0:
        msk = torch.empty(w.N, dtype=torch.uint8, device=dev)
        mlist = np.ascontiguousarray(w.modes[:, 1])
        F.few_mode_select(ctx.handle, dev_in[2], dev_in[3], mlist, 1e-5, msk, sh)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(10)]
        for a, b_ in evs:
            a.record(stream)
            F.few_mode_select(ctx.handle, dev_in[2], dev_in[3], mlist, 1e-5, msk, sh)
            b_.record(stream)
        torch.cuda.synchronize()
        selector = {"ms": sum(a.elapsed_time(b_) for a, b_ in evs) / len(evs), "eps": 1e-5,
                    "knots": w.K, "modes": w.N, "selected": int(msk.sum().item())}

    # direct (non-interpolated) summation over dense arrays: HBM-bound in mixed precision
    direct = None
    if rank == 0 and args.direct_samples > 0:
        nsd = args.direct_samples
        tsd = torch.arange(nsd, dtype=torch.float64, device=dev) * w.dt + 1.0e6
        xd = (tsd / w.T)[:, None]
        am = w.amp_model
        ta = lambda a: torch.as_tensor(a, device=dev)[None, :]
        env = ta(am.a) * (1.0 + ta(am.alpha) * xd + ta(am.beta) * xd * xd)
        d_re = (env * torch.cos(ta(am.psi))).contiguous()
        d_im = (env * torch.sin(ta(am.psi))).contiguous()
        del env
        d_pp = torch.as_tensor(W.phase_phi(tsd.cpu().numpy(), w.T, w.phi_phi0), device=dev)
        d_pr = torch.as_tensor(W.phase_r(tsd.cpu().numpy(), w.T, w.phi_r0), device=dev)
        d_out = torch.empty(nsd, dtype=torch.complex64, device=dev)
        F.few_direct_sum(ctx.handle, d_pp, d_pr, d_re, d_im, w.modes, w.theta, w.phi, d_out,
                         1.0, F.FEW_MIXED, sh)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(5)]
        for a, b_ in evs:
            a.record(stream)
            F.few_direct_sum(ctx.handle, d_pp, d_pr, d_re, d_im, w.modes, w.theta, w.phi, d_out,
                             1.0, F.FEW_MIXED, sh)
            b_.record(stream)
        torch.cuda.synchronize()
        msd = min(a.elapsed_time(b_) for a, b_ in evs)
        nbytes = nsd * (16 * w.N + 16 + 8)
        gbs = nbytes / (msd * 1e-3) / 1e9
        hbm = float(_peaks_file().get("hbm_gbs", 6800.0))
        direct = {"samples": nsd, "modes": w.N, "ms": msd,
                  "mode_samples_per_s": nsd * w.N / (msd * 1e-3),
                  "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                               "frac": gbs / hbm, "bytes_per_launch": nbytes,
                               "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}}
        del d_re, d_im, d_pp, d_pr, d_out

    # reduced-basis amplitudes (Sec. 3.E): 99 coefficients per knot -> 3843 modes, for the knots
    # of many trajectories at once, renormalised; the output (FP64 amplitudes) is what the
    # spline build reads
    rb = None
    if rank == 0 and args.rb_knots > 0:
        rb = bench_rb(ctx, args.rb_knots, w.N, stream, sh)

    # pipe peaks
    peaks = measure_peaks(local_rank) if rank == 0 and not args.no_probe else {}

    torch.cuda.synchronize()
    tr.release()
    ctx.close()
    return dict(w=w, ms_local=ms_local, step_ms=step_ms, kernel_ms=kernel_ms, last_t=last_t,
                clocks=clocks, plain=plain, e2e=e2e, peaks=peaks, slots=slots,
                h_fast=h_fast, h_plain=h_plain, prec=prec, batched=batched, tile=tile,
                selector=selector, direct=direct, rb=rb)


def run_serving(args):
    """Serving workload: Poisson MCMC-like stream at 50/90/120% of the measured capacity."""
    import torch
    from paper_2104_04582_gb300 import _build
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT
    from paper_2104_04582_gb300.serve import GpuEngine, Request, Server

    _build.build()
    torch.cuda.set_device(0)
    n_req = args.serving_requests
    trajs_in, stream = W.config4_stream(n_req, rate_hz=1.0)
    ctx = RT.Context(0)
    trajs = {k: RT.from_inputs(ctx, w) for k, w in trajs_in.items()}

    def reqs_for(prec):
        out = []
        for r in stream:
            w = trajs_in[r.traj_key]
            out.append(Request(traj_key=r.traj_key, n_samples=w.n_samples, dt=w.dt, t0=w.t0,
                               theta=r.theta, phi=r.phi, scale=r.scale, dphi_phi0=r.dphi_phi0,
                               dphi_r0=r.dphi_r0, prec=prec))
        return out

    def run(reqs, rate_hz=None, seed=0):
        srv = Server(GpuEngine(ctx, trajs), hbm_budget_bytes=int(args.serving_budget_gb * 2 ** 30),
                     max_batch=16, max_inflight=3)
        rng = np.random.default_rng(seed)
        t0 = time.perf_counter()
        t_arr = 0.0
        futs = []
        for r in reqs:
            if rate_hz:
                t_arr += float(rng.exponential(1.0 / rate_hz))
                d = t_arr - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
            futs.append(srv.submit(r))
        srv.drain()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        for f in futs:
            f.result()
        st["wall_s"] = wall
        st["offered_rate_hz"] = rate_hz
        return st

    mixed = reqs_for(F.FEW_MIXED)
    run(mixed[:16])  # warm-up
    burst = run(mixed)
    cap = burst["completed"] / burst["wall_s"]
    loads = {}
    for f in (0.5, 0.9, 1.2):
        loads[f"{int(f * 100)}%"] = run(mixed, rate_hz=f * cap, seed=int(f * 100))
    plain = run(reqs_for(F.FEW_FP64)[:max(8, n_req // 10)])
    torch.cuda.synchronize()
    samples = [trajs_in[r.traj_key].n_samples for r in stream]
    modes = [trajs_in[r.traj_key].N for r in stream]
    line = {"mode": "serving", "metric": "waveforms/s and p50/p99 latency, Poisson MCMC-like stream",
            "unit": "waveforms/s", "n_gpus": 1, "requests": n_req,
            "config": {"workload": "requests of 0.5-4 yr, dt in {5,10,15} s, 10-1000 modes, "
                                   "perturbed angles/phases/scale of resident trajectories, "
                                   "10% new trajectories", "seed": W.SEEDS["C4"],
                       "trajectories": len(trajs), "mean_samples": float(np.mean(samples)),
                       "mean_modes": float(np.mean(modes)),
                       "budget_gb": args.serving_budget_gb, "max_batch": 16, "max_inflight": 3},
            "capacity_mixed": {"value": cap, "p50_ms": burst["p50_ms"], "p99_ms": burst["p99_ms"]},
            "loads": {k: {"offered_hz": v["offered_rate_hz"], "waveforms_per_s": v["waveforms_per_s"],
                          "p50_ms": v["p50_ms"], "p99_ms": v["p99_ms"],
                          "max_inflight_batches": v["max_inflight_batches"]}
                      for k, v in loads.items()},
            "plain_fp64_capacity": {"value": plain["completed"] / plain["wall_s"],
                                    "requests": plain["completed"]}}
    line["capacity_vs_plain_fp64"] = cap / line["plain_fp64_capacity"]["value"]
    for tr in trajs.values():
        tr.release()
    ctx.close()
    print(json.dumps(line))
    return 0


def run_profile_case(which: str, repeats: int = 3) -> int:
    """A short, untimed run of the benchmark workload for profiler captures: the one-year
    3843-mode waveform computed `repeats` times (the first launch of each kernel is warm-up)."""
    import torch
    from paper_2104_04582_gb300 import _build
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT
    _build.build()
    prec = F.FEW_FP64 if which == "fp64" else F.FEW_MIXED
    w = W.config2()
    if which == "select":
        # Mode Selector over the one-year workload's knots: 100 knots x 3843 modes, eps = 1e-5
        dev = torch.device("cuda", 0)
        are = torch.as_tensor(np.ascontiguousarray(w.amp_re)).to(dev)
        aim = torch.as_tensor(np.ascontiguousarray(w.amp_im)).to(dev)
        mask = torch.empty(w.N, dtype=torch.uint8, device=dev)
        with RT.Context(0) as ctx:
            for _ in range(repeats):
                F.few_mode_select(ctx.handle, are, aim, w.modes[:, 1], 1e-5, mask, RT.current_stream())
            torch.cuda.synchronize()
            st = ctx.sync_status()
        print(json.dumps({"profile_case": which, "repeats": repeats, "status": int(st)}))
        return 0 if st == F.FEW_OK else 1
    if which == "rb":
        # 6400 knots (64 trajectories x 100), 99 coefficients, 3843 modes, mixed, renormalised
        dev = torch.device("cuda", 0)
        (are, aim), (bre, bim), nu = _rb_device_inputs(6400, w.N, 64, dev)
        ore = torch.empty((6400, w.N), dtype=torch.float64, device=dev)
        oim = torch.empty_like(ore)
        with RT.Context(0) as ctx:
            h = F.few_basis_create(ctx.handle, bre, bim, RT.current_stream())
            for _ in range(repeats):
                F.few_rb_amplitudes(ctx.handle, h, are, aim, ore, oim, nu, F.FEW_MIXED,
                                    RT.current_stream())
            torch.cuda.synchronize()
            st = ctx.sync_status()
            F.few_basis_release(ctx.handle, h)
        print(json.dumps({"profile_case": which, "repeats": repeats, "status": int(st)}))
        return 0 if st == F.FEW_OK else 1
    if which == "direct":
        # 30,000 samples x 3843 modes of dense FP64 amplitudes (1.8 GB, larger than L2)
        ts = w.t0 + (np.arange(30000) + 1000000) * w.dt
        pphi, pr = w.phases_at(ts)
        A = w.amp_model(ts)
        dev = [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in (pphi, pr, A.real, A.imag)]
        out = torch.empty(len(ts), dtype=torch.complex64, device="cuda")
        with RT.Context(0) as ctx:
            for _ in range(repeats):
                F.few_direct_sum(ctx.handle, *dev, w.modes, w.theta, w.phi, out, 1.0, F.FEW_MIXED,
                                 RT.current_stream())
            torch.cuda.synchronize()
            st = ctx.sync_status()
        print(json.dumps({"profile_case": which, "repeats": repeats, "status": int(st)}))
        return 0 if st == F.FEW_OK else 1
    with RT.Context(0) as ctx:
        tr = RT.from_inputs(ctx, w)
        for _ in range(repeats):
            RT.waveform_inputs(ctx, tr, w, prec)
        torch.cuda.synchronize()
        st = ctx.sync_status()
        tr.release()
    print(json.dumps({"profile_case": which, "repeats": repeats, "status": int(st)}))
    return 0 if st == F.FEW_OK else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--rb-knots", type=int, default=6400,
                    help="knots of the reduced-basis amplitude measurement (0: skip)")
    ap.add_argument("--profile-case", choices=["mixed", "fp64", "direct", "rb", "select"], default=None,
                    help="untimed runs of the benchmark waveform for profiler captures")
    ap.add_argument("--serving", action="store_true",
                    help="run the serving workload instead of the single-waveform benchmark")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--serving-budget-gb", type=float, default=16.0)
    ap.add_argument("--direct-samples", type=int, default=100000,
                    help="samples of the direct-summation measurement (0: skip)")
    ap.add_argument("--batch", type=int, default=8,
                    help="waveforms per step of the batched-path measurement (0: skip)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.profile_case:
        return run_profile_case(args.profile_case)

    if args.serving and args.impl != "reference":
        return run_serving(args) if rank == 0 else 0

    if args.impl == "reference":
        if rank != 0:
            return 0
        w = W.config2()
        per_step = []
        cb = None
        vals = []
        for k in range(args.warmup + args.steps):
            cb, _ = cpu_baseline(w, target_s=max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps))))
            if k >= args.warmup:
                vals.append(cb["value"])
        v = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "seed": W.SEEDS["C2"],
                           "note": "each step times the oracle on a bounded prefix of the waveform"},
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    res = run_gpu(args, rank, world, local_rank)
    ms = res["ms_local"]
    if world > 1:
        import torch
        import torch.distributed as dist
        ms = dist_max(ms, torch.device("cuda", local_rank))
        dist.barrier()
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    w = res["w"]
    value = aggregate_value(ms, world)  # every rank computed one waveform per step
    mode_samples = w.N * w.n_samples
    slots = res["slots"]
    kms = statistics.mean(res["kernel_ms"]) if res["kernel_ms"] else float("nan")
    fp32 = res["prec"] == 1
    # algorithmic arithmetic of the summation kernel: one complex cubic (6 FMA) and one complex
    # Horner step (4 FMA) per (harmonic slot, sample); an FMA is 2 flops
    flops = 20.0 * slots * w.n_samples
    achieved = flops / (kms * 1e-3) / 1e12
    clocks = res["clocks"] or {}
    mp = _peaks_file()
    sm_max = float(mp.get("sm_max_mhz", 2070.0))
    if fp32:
        peak = N_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        peak_src = (f"FP32 FMA: {N_SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {sm_max:.0f} MHz "
                    "(max SM clock)")
    else:
        peak = FP64_NOMINAL_TFLOPS
        peak_src = "FP64 nominal 1.25 TFLOP/s"
    probe = res["peaks"]
    traffic = None
    if fp32 and _kernel_source_hash() == PROFILED_TRAFFIC["source_sha256_16"] and             res.get("tile") == PROFILED_TRAFFIC["tile"]:
        traffic = PROFILED_TRAFFIC["bytes"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
            "kernel": "k_sum<float,R> (mixed)" if fp32 else "k_sum<double,R> (fp64)",
            "kernel_ms": kms, "flops_per_launch": flops,
            "peak_source": peak_src}
    if probe:
        key = "fp32_fma_per_s" if fp32 else "fp64_fma_per_s"
        if key in probe:
            pm = 2 * probe[key] / 1e12
            roof["peak_probe_tflops"] = pm
            roof["frac_of_probe"] = achieved / pm
        if fp32 and "fp32_fma_3reg_per_s" in probe:
            # the Horner loop's FMAs take three register operands: the measured rate of that
            # instruction form is the ceiling the kernel can reach
            p3 = 2 * probe["fp32_fma_3reg_per_s"] / 1e12
            roof["peak_register_operand_tflops"] = p3
            roof["frac_of_register_operand_rate"] = achieved / p3
        if fp32 and "fp32_fma_summation_block_per_s" in probe:
            # the kernel's own per-slot block (coefficients from shared memory, two cubics, the
            # complex step) run in isolation: what the inner loop can reach on this chip
            pb = 2 * probe["fp32_fma_summation_block_per_s"] / 1e12
            roof["peak_summation_block_tflops"] = pb
            roof["frac_of_summation_block_rate"] = achieved / pb
    if clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = achieved / (peak * clocks["sm_mhz"] / sm_max)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if fp32 else "f64",
        "precision": ("mixed: FP64 phase splines and mod-2pi reduction; FP32 amplitudes, "
                      "exponential powers and accumulation") if fp32 else "fp64 throughout",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "seed": W.SEEDS["C2"], "knots": w.K, "modes": w.N,
                   "samples": w.n_samples, "harmonic_slots": slots,
                   "l2": "flushed (256 MB write) between timed steps",
                   "step": "spline build + harmonics + fold + mode sum, inputs resident in HBM",
                   "parallelism": f"replicas x{world}"},
        "mode_samples_per_s": world * mode_samples / (ms * 1e-3),
        "kernel_ms": {"build": res["last_t"][0], "harmonics": res["last_t"][1],
                      "fold": res["last_t"][2], "sum": kms},
        "roofline": roof,
        "gpu_launches": 4 * args.steps,
        "clocks": clocks or None,
        "e2e": res["e2e"],
    }
    if res["plain"]:
        line["plain_fp64"] = res["plain"]
        line["speedup_vs_plain_fp64"] = res["plain"]["ms_per_step"] / ms
    if res.get("direct"):
        line["direct_sum"] = res["direct"]
    if res.get("rb"):
        line["rb_amplitudes"] = res["rb"]
    if res.get("selector"):
        line["mode_selector"] = res["selector"]
    if res.get("batched"):
        line["batched"] = res["batched"]
        if res["plain"]:
            line["batched"]["speedup_vs_plain_fp64"] = res["batched"]["value"] / res["plain"]["value"]
    if probe:
        line["measured_pipe_peaks"] = {k: v for k, v in probe.items()}
    # accuracy of this run's outputs
    acc = {}
    if res["h_plain"] is not None:
        acc["mismatch_mixed_vs_fp64_full_series"] = _mismatch(res["h_fast"], res["h_plain"])
    if not args.no_cpu:
        cb, h_or = cpu_baseline(w, target_s=args.cpu_seconds)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        import oracle
        n = len(h_or)
        acc["mismatch_vs_oracle_window"] = oracle.mismatch(res["h_fast"][:n], h_or)
        acc["rel_l2_vs_oracle_window"] = float(np.linalg.norm(res["h_fast"][:n] - h_or)
                                               / np.linalg.norm(h_or))
        if res["h_plain"] is not None:
            hp = res["h_plain"]
            acc["fp64_rel_l2_vs_oracle_window"] = float(np.linalg.norm(hp[:n] - h_or)
                                                        / np.linalg.norm(h_or))
        acc["oracle_window_samples"] = n
    line["accuracy"] = acc
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
