#!/usr/bin/env python3
"""Benchmark of the interpolated EMRI mode summation on GB300.

Headline workload (the configuration the metric is quoted on): one 1-yr waveform at dt = 10 s
(3,155,760 samples), K = 100 knots, the full 3843-mode Schwarzschild grid (l = 2..10,
m = 0..l, n = -30..30), synthetic seeded inputs.  A step is one pass of the whole hot path
with the knot data resident in HBM: spline build (all 7688 splines), harmonics, fold, phase
anchors and the per-sample mode sum, written to a device buffer.

Default arm (--impl gb300): the mixed-precision path; beside it, on the same GPU and in the same
JSON line: the plain FP64 path on the same waveform, the end-to-end call with host buffers, the
256-waveform batch (one persistent launch replayed as a CUDA graph), the serving loop on a
Poisson request stream at 50/90/120 % of its measured capacity (p50/p99 latency), the 4-yr
stress waveform, and the Mode Selector, direct-summation and reduced-basis kernels.
Reference arm (--impl reference): the FP64 CPU oracle on the host cores, on a bounded sample of
the same workload, same metric.

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
# one that was profiled (hash of the code of sum.cu + phase_eval.cuh + async.cuh, comments
# left out) and the launch shape (R, threads) is the profiled one.  The stage size is left out: it changes how the L2-resident slot
# tables are staged, not which bytes come from DRAM (the tables and anchors once, the output
# still in L2 when the launch ends).
PROFILED_TRAFFIC = {"source_sha256_16": "c81bdd4aa4270df9", "tile": (8, 256), "bytes": 13583360 + 0}
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (4 sub-partitions x 32)
FP64_FMA_PER_SM_CLK = 2   # FP64 FMA per SM per clock on GB300 (1.25 TFLOP/s at 152 SMs, 2.07 GHz)


def device_peaks(dev_index: int) -> dict:
    """Nominal FP32 / FP64 FMA peaks of this device: its SM count (queried) x lanes x 2 flop x
    the maximum SM clock (measured peaks file, else the GPU's own report)."""
    import torch
    sms = int(torch.cuda.get_device_properties(dev_index).multi_processor_count)
    mhz = float(_peaks_file().get("sm_max_mhz", 0.0))
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", f"--id={dev_index}", "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                 timeout=20)
            mhz = float(out.stdout.strip().splitlines()[0])
        except (OSError, ValueError, IndexError, subprocess.SubprocessError):
            mhz = 2070.0
    return {"sms": sms, "sm_max_mhz": mhz,
            "fp32_tflops": sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
            "fp64_tflops": sms * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12,
            "source": f"{sms} SMs (device query) x lanes x 2 flop x {mhz:.0f} MHz"}


def _code_hash(paths) -> str:
    """Hash of the code in C/CUDA sources: line comments, trailing blanks and blank lines left
    out, so that a comment edit keeps the hash while any code change alters it."""
    import hashlib
    import re
    h = hashlib.sha256()
    for p in paths:
        with open(p, encoding="utf-8") as fh:
            for line in fh:
                code = re.sub(r"//.*$", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _kernel_source_hash() -> str:
    """Code hash of the summation kernel's sources (the key of a profiled traffic figure)."""
    d = os.path.join(ROOT, "paper_2104_04582_gb300", "csrc")
    return _code_hash([os.path.join(d, f) for f in ("sum.cu", "phase_eval.cuh", "async.cuh")])


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

def cpu_baseline(w, target_s: float = 12.0, max_samples=None, threads=None,
                 what: str = "the 1-yr 3843-mode waveform"):
    """The oracle, as it stands, on a bounded prefix of the workload, on `threads` host threads
    (default: all host cores).

    A call costs a fixed part (all splines and harmonics) plus a part per sample; two short calls
    fit both, a third call of about `target_s` measures the per-sample rate, and the whole
    waveform's time is extrapolated as fixed + rate x N_s (no extrapolation when the third call
    covers every sample).
    """
    import oracle
    threads = int(threads or os.cpu_count() or 1)

    def run(n):
        t0 = time.perf_counter()
        h = oracle.waveform_inputs(w, 0, n, nthreads=threads)
        return time.perf_counter() - t0, h

    n2 = min(2048, w.n_samples)
    n1 = max(1, min(256, n2 // 8))
    t1, _ = run(n1)
    t2, _ = run(n2)
    per = max((t2 - t1) / max(n2 - n1, 1), 1e-12)
    fixed = max(t1 - per * n1, 0.0)
    n = int(min(w.n_samples, max(n2, (target_s - fixed) / per)))
    if max_samples:
        n = min(n, max_samples)
    el, h = run(n)
    per = max((el - fixed) / n, 1e-12)
    t_full = fixed + per * w.n_samples
    rate = n * w.N / max(el - fixed, 1e-9)
    if n >= w.n_samples:
        t_full = el
        rate = n * w.N / max(el, 1e-9)
        how = f"all {n} samples of {what} ({n * w.N:.3g} mode-samples) in {el:.2f} s on {threads} " \
              f"OpenMP threads"
    else:
        how = (f"first {n} of {w.n_samples} samples of {what} ({n * w.N:.3g} mode-samples) in "
               f"{el:.1f} s on {threads} OpenMP threads; fixed cost {fixed:.2f} s + "
               f"{per * 1e6:.1f} us/sample extrapolated to the whole waveform ({t_full:.0f} s)")
    return {"value": 1.0 / t_full, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": how, "mode_samples_per_s": rate, "seconds": el,
            "seconds_full_waveform": t_full}, h


def cpu_baseline_detail(w, target_s: float = 3.0) -> dict:
    """The oracle's rate on one host thread and on all of them: the one-year waveform `w` on
    one thread (a bounded prefix, extrapolated like cpu_baseline), the one-week 132-mode
    waveform in full on all cores and on one."""
    keep = ("value", "unit", "cores", "sample", "mode_samples_per_s", "seconds_full_waveform")
    out = {}
    cb, _ = cpu_baseline(w, target_s=target_s, threads=1)
    out["one_year_single_thread"] = {k: cb[k] for k in keep}
    w1 = W.config1()
    for key, thr in (("one_week_all_cores", None), ("one_week_single_thread", 1)):
        cb, _ = cpu_baseline(w1, target_s=target_s, threads=thr,
                             what="the 1-week 132-mode waveform")
        out[key] = {k: cb[k] for k in keep}
    return out


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


def _timed(stream, fn, reps, flush=None):
    """Per-rep device time (ms) of fn() queued on `stream`, CUDA events on that stream, the L2
    flushed (outside the events) before every rep when a flush buffer is given."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    for a, b in evs:
        if flush is not None:
            flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


IN_FLIGHT_SETS = 5  # rotating sets of ~60 MB each (knot data, spline data, output): > L2


def _in_flight(ctx, sets, streams, steps):
    """`steps` one-waveform steps (spline build + waveform), step j on stream j % len(streams)
    with set j % len(sets); a set's next use waits for its previous one.  Returns the device time
    (ms) from an event before the first step to one after the last, on the current stream."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    cur = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(cur)
    for s in streams:
        s.wait_event(a)
    done = [None] * len(sets)
    for j in range(steps):
        s, k = streams[j % len(streams)], j % len(sets)
        tr, dev_in, out, req = sets[k]
        if done[k] is not None:
            s.wait_event(done[k])
        h = int(s.cuda_stream)
        F.few_traj_set_data(ctx.handle, tr.handle, *dev_in, stream=h)
        F.few_waveform(ctx.handle, req, h)
        done[k] = torch.cuda.Event()
        done[k].record(s)
    for s in streams:
        cur.wait_stream(s)
    b.record(cur)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def bench_step_c2(args, ctx, w, dev, stream, sh, flush, prec, rank, world, tune_cache):
    """The headline step on the one-year workload: spline build + harmonics + fold + anchors +
    mode sum, knot data resident in HBM, timed with `args.in_flight` waveforms in flight (also
    timed one at a time, L2 flushed before each).  Returns the timed steps and kernel figures."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT
    from paper_2104_04582_gb300 import tune

    c64 = prec == F.FEW_MIXED
    tr = RT.Trajectory(ctx, w.t_knots, w.modes)
    dev_in = tr.upload_inputs(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
    out = RT.alloc_out(w.n_samples, c64, dev.index)
    req = RT.request(tr, out, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec)
    K_, N_, slots = tr.info

    def step():
        F.few_traj_set_data(ctx.handle, tr.handle, *dev_in, stream=sh)
        F.few_waveform(ctx.handle, req, sh)

    step()
    torch.cuda.synchronize()
    tile, tuned_now = tune.ensure(ctx.handle, lambda: F.few_waveform(ctx.handle, req, sh), prec,
                                  slots, w.n_samples, tune_cache)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("device error during warm-up")

    F.few_ctx_set_timing(ctx.handle, False)  # no per-kernel events inside the timed steps
    # one waveform at a time: every step alone on the stream, L2 flushed before each
    seq_ms = _timed(stream, step, args.steps, flush)
    # the headline: `in_flight` waveforms in flight on as many streams, each step on one of
    # IN_FLIGHT_SETS rotating (trajectory, knot data, output) sets, whose working set exceeds L2
    sets, streams = [], []
    if args.in_flight > 1:
        sets = [(tr, dev_in, out, req)]
        for _ in range(IN_FLIGHT_SETS - 1):
            t_ = RT.Trajectory(ctx, w.t_knots, w.modes)
            d_ = t_.upload_inputs(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
            o_ = RT.alloc_out(w.n_samples, c64, dev.index)
            sets.append((t_, d_, o_, RT.request(t_, o_, w.n_samples, w.t0, w.dt, w.theta,
                                                 w.phi, prec)))
        streams = [torch.cuda.Stream(device=dev) for _ in range(args.in_flight)]
        _in_flight(ctx, sets, streams, args.warmup)
        torch.cuda.synchronize()
    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sets:
        total = _in_flight(ctx, sets, streams, args.steps)
        step_ms = [total / args.steps] * args.steps
    else:
        step_ms = _timed(stream, step, args.steps, flush)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    for t_, _, _, _ in sets[1:]:
        t_.release()
    del sets
    # the kernels' own durations: the library's event pairs on the launch stream, read after
    # each of a few more flushed steps (reading waits for the step, so outside the timed loop)
    F.few_ctx_set_timing(ctx.handle, True)
    kt = []
    for _ in range(min(args.steps, 5)):
        flush.zero_()
        step()
        kt.append(F.few_last_timing(ctx.handle))
    F.few_ctx_set_timing(ctx.handle, False)
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("device error during the timed region")
    h = out.cpu().numpy().astype(np.complex128) if rank == 0 else None
    res = dict(tr=tr, dev_in=dev_in, step_ms=step_ms, seq_ms=seq_ms, clocks=clocks, h=h,
               slots=slots,
               tile=tuple(tile), tile_tuned_now=tuned_now,
               kernel_ms={"build": statistics.median(k[0] for k in kt),
                          "harmonics": statistics.median(k[1] for k in kt),
                          "fold_and_anchors": statistics.median(k[2] for k in kt),
                          "sum": statistics.median(k[3] for k in kt)},
               sum_ms=[float(k[3]) for k in kt if k[3] > 0])
    del out
    return res


def bench_plain_fp64(ctx, w, tr, dev_in, dev, stream, sh, flush, reps):
    """The plain FP64 path on the same waveform (every step FP64)."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT
    out64 = RT.alloc_out(w.n_samples, False, dev.index)
    req64 = RT.request(tr, out64, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_FP64)

    def step():
        F.few_traj_set_data(ctx.handle, tr.handle, *dev_in, stream=sh)
        F.few_waveform(ctx.handle, req64, sh)

    step()
    torch.cuda.synchronize()
    ms = _timed(stream, step, reps, flush)
    F.few_ctx_set_timing(ctx.handle, True)
    step()
    sum64 = F.few_last_timing(ctx.handle)[3]
    F.few_ctx_set_timing(ctx.handle, False)
    h64 = out64.cpu().numpy()
    m = statistics.mean(ms)
    return {"ms_per_step": m, "value": 1000.0 / m, "unit": UNIT, "steps": reps,
            "mode_samples_per_s": w.N * w.n_samples / (m * 1e-3), "sum_kernel_ms": sum64,
            "dtype": "f64"}, h64


def bench_e2e(ctx, w, tr, prec, sh, flush, steps, in_flight=1):
    """End to end through the C ABI: pinned host knot data in, pinned host output out, both
    copies inside the timed region (host wall clock around the two calls).  With in_flight > 1,
    as many host threads make the same calls at once, each with its own trajectory, host
    buffers and stream (the library does not hold the context while a call waits for its
    copies or its result); value = all their steps / wall time."""
    import threading
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT
    c64 = prec == F.FEW_MIXED
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    def make(tr_):
        h_in = [pin(a) for a in (w.phi_phi, w.phi_r, w.amp_re, w.amp_im)]
        host_out = torch.empty(w.n_samples, dtype=torch.complex64 if c64 else torch.complex128
                               ).pin_memory().numpy()
        req = RT.request(tr_, host_out, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec,
                         out_where=F.FEW_MEM_HOST)
        return tr_, h_in, host_out, req

    def one(st, s_):
        tr_, h_in, _, req = st
        F.few_traj_set_data(ctx.handle, tr_.handle, *h_in, stream=s_)
        F.few_waveform(ctx.handle, req, s_)  # host output: returns once the result is in host memory

    main = make(tr)
    for _ in range(2):
        one(main, sh)
    torch.cuda.synchronize()
    t_e = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one(main, sh)
        t_e.append(time.perf_counter() - t0)
    res = {"value": 1.0 / statistics.mean(t_e), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(a.nbytes for a in main[1])),
           "d2h_bytes_per_step": int(main[2].nbytes),
           "ms_per_step": 1000.0 * statistics.mean(t_e), "steps": steps,
           "timer": "host wall clock around the two C-ABI calls (the call with host output "
                    "returns once the result is in host memory; page-locked output is stored by "
                    "the summation kernel directly)"}
    if in_flight > 1:
        extra = [RT.Trajectory(ctx, w.t_knots, w.modes) for _ in range(in_flight - 1)]
        sets = [main] + [make(t_) for t_ in extra]
        streams = [torch.cuda.Stream() for _ in sets]
        per = max(2, steps)
        go = threading.Barrier(len(sets) + 1)
        errs = []

        def worker(st, strm):
            try:
                one(st, int(strm.cuda_stream))  # warm-up of this thread's set
                go.wait()
                for _ in range(per):
                    one(st, int(strm.cuda_stream))
            except Exception as e:  # noqa: BLE001 -- reported below
                errs.append(e)
                go.abort()
        ths = [threading.Thread(target=worker, args=(st, strm)) for st, strm in zip(sets, streams)]
        for th in ths:
            th.start()
        try:
            go.wait()
        except threading.BrokenBarrierError:
            pass  # a worker failed before the start; its error is raised below
        t0 = time.perf_counter()
        for th in ths:
            th.join()
        wall = time.perf_counter() - t0
        for t_ in extra:
            t_.release()
        if errs:
            raise errs[0]
        seq = dict(res)
        res = {"value": per * len(sets) / wall, "unit": UNIT,
               "h2d_bytes_per_step": seq["h2d_bytes_per_step"],
               "d2h_bytes_per_step": seq["d2h_bytes_per_step"],
               "ms_per_step": 1000.0 * wall / (per * len(sets)), "steps": per * len(sets),
               "in_flight": len(sets),
               "timer": "host wall clock from a barrier before the first step of %d host "
                        "threads to the end of the last; each thread makes the two C-ABI calls "
                        "per step with its own trajectory, pinned buffers and stream" % len(sets),
               "sequential": {k: seq[k] for k in ("value", "ms_per_step", "steps", "timer")}}
    return res


C2_SLOT_SAMPLES = 1281 * 3155760  # slots x samples of the one-year 3843-mode waveform
C2_MODE_SAMPLES = 3843 * 3155760


def bench_batched_c3(ctx, dev, stream, sh, flush, n_waves, reps, tune_cache, oracle_windows=4,
                     in_flight=1):
    """256 waveforms of 0.25-2 yr, K 50-150, power-selected 10-3843 modes, mixed precision:
    spline rebuild of every trajectory + harmonics + fold + anchors + one persistent summation
    launch, captured once as a CUDA graph and replayed; tile chosen by the autotuner on a
    16-waveform sub-batch."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT
    from paper_2104_04582_gb300 import tune
    import oracle
    t_in = time.perf_counter()
    ws = W.config3(n_waves)
    trs = [RT.from_inputs(ctx, x) for x in ws]
    outs = [RT.alloc_out(x.n_samples, True, dev.index) for x in ws]
    reqs = [RT.request(t_, o_, x.n_samples, x.t0, x.dt, x.theta, x.phi, F.FEW_MIXED)
            for t_, o_, x in zip(trs, outs, ws)]
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_in
    sub = reqs[:16]
    sub_slots = max(t_.info[2] for t_ in trs[:16])
    sub_samples = sum(x.n_samples for x in ws[:16])
    tile, tuned_now = tune.ensure(
        ctx.handle, lambda b: F.few_batch_run(ctx.handle, b, sh), F.FEW_MIXED, sub_slots,
        sub_samples, tune_cache,
        prepare=lambda: F.few_batch_plan(ctx.handle, sub, F.FEW_BATCH_NO_GRAPH),
        cleanup=lambda b: (torch.cuda.synchronize(), F.few_batch_release(ctx.handle, b)))
    t_plan = time.perf_counter()
    bh = F.few_batch_plan(ctx.handle, reqs, F.FEW_BATCH_REBUILD_SPLINES)
    plan_s = time.perf_counter() - t_plan
    for _ in range(2):
        F.few_batch_run(ctx.handle, bh, sh)
    torch.cuda.synchronize()
    ms = _timed(stream, lambda: F.few_batch_run(ctx.handle, bh, sh), reps, flush)
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("device error in the batched run")
    msb = statistics.mean(ms)
    flight = None
    if in_flight > 1:
        # more batches in flight: each its own trajectories, outputs and graph, on its own stream
        sets = [(bh, None, None)]
        for _ in range(in_flight - 1):
            trs2 = [RT.from_inputs(ctx, x) for x in ws]
            outs2 = [RT.alloc_out(x.n_samples, True, dev.index) for x in ws]
            reqs2 = [RT.request(t_, o_, x.n_samples, x.t0, x.dt, x.theta, x.phi, F.FEW_MIXED)
                     for t_, o_, x in zip(trs2, outs2, ws)]
            sets.append((F.few_batch_plan(ctx.handle, reqs2, F.FEW_BATCH_REBUILD_SPLINES), trs2,
                         outs2))
        streams = [torch.cuda.Stream(device=dev) for _ in sets]
        for (b_, _, _), s_ in zip(sets, streams):
            F.few_batch_run(ctx.handle, b_, int(s_.cuda_stream))
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(cur)
        for s_ in streams:
            s_.wait_event(a)
        for _ in range(reps):
            for (b_, _, _), s_ in zip(sets, streams):
                F.few_batch_run(ctx.handle, b_, int(s_.cuda_stream))
        for s_ in streams:
            cur.wait_stream(s_)
        e.record(cur)
        torch.cuda.synchronize()
        tot = a.elapsed_time(e)
        if ctx.sync_status() != F.FEW_OK:
            raise RuntimeError("device error in the batched run")
        nb = reps * len(sets)
        flight = {"batches_in_flight": len(sets), "batches": nb, "ms_per_batch": tot / nb,
                  "value": n_waves * nb * 1000.0 / tot, "unit": "waveforms/s",
                  "note": "each batch with its own 256 trajectories, outputs and graph, replayed "
                          "on its own stream; CUDA events from before the first batch to after "
                          "the last"}
        for b_, trs2, outs2 in sets[1:]:
            F.few_batch_release(ctx.handle, b_)
            for t_ in trs2:
                t_.release()
            del outs2
    samples = sum(x.n_samples for x in ws)
    mode_samples = sum(x.N * x.n_samples for x in ws)
    slot_samples = sum(t_.info[2] * x.n_samples for t_, x in zip(trs, ws))
    # accuracy: the oracle on a 2000-sample window in the middle of a few of the waveforms
    acc = []
    for q in np.linspace(0, n_waves - 1, oracle_windows).astype(int):
        x = ws[q]
        i0 = max(0, x.n_samples // 2 - 1000)
        n = min(2000, x.n_samples - i0)
        o = oracle.waveform_inputs(x, i0, n, nthreads=os.cpu_count() or 1)
        g = outs[q][i0:i0 + n].cpu().numpy().astype(np.complex128)
        acc.append({"waveform": int(q), "modes": int(x.N), "window": [int(i0), int(n)],
                    "mismatch_vs_oracle": oracle.mismatch(g, o),
                    "rel_l2_vs_oracle": float(np.linalg.norm(g - o) / np.linalg.norm(o))})
    res = {"waveforms_per_step": n_waves, "ms_per_step": msb, "steps": reps,
           "value": n_waves * 1000.0 / msb, "unit": "waveforms/s",
           "samples_per_s": samples / (msb * 1e-3),
           "mode_samples_per_s": mode_samples / (msb * 1e-3),
           "slot_samples_per_s": slot_samples / (msb * 1e-3),
           "c2_equivalent_waveforms_per_s_by_mode_samples": mode_samples / C2_MODE_SAMPLES / (msb * 1e-3),
           "c2_equivalent_waveforms_per_s_by_slot_samples": slot_samples / C2_SLOT_SAMPLES / (msb * 1e-3),
           "total_samples": samples, "total_mode_samples": mode_samples,
           "modes_min_median_max": [int(min(x.N for x in ws)), int(statistics.median(x.N for x in ws)),
                                    int(max(x.N for x in ws))],
           "tile": list(tile), "tile_tuned_in_this_run": tuned_now,
           "launches_per_step": 5, "graph": True, "precision": "mixed",
           "step": "spline rebuild of all 256 trajectories + harmonics + fold + phase anchors + "
                   "one persistent summation launch, replayed as one CUDA graph",
           "host_setup_s": setup_s, "plan_and_capture_s": plan_s, "accuracy": acc}
    if flight:
        flight["slot_samples_per_s"] = slot_samples * flight["value"] / n_waves
        flight["c2_equivalent_waveforms_per_s_by_slot_samples"] = \
            slot_samples / C2_SLOT_SAMPLES * flight["value"] / n_waves
        res["in_flight"] = flight
    F.few_batch_release(ctx.handle, bh)
    for t_ in trs:
        t_.release()
    del outs
    torch.cuda.synchronize()
    return res


def bench_stress_c5(ctx, dev, stream, sh, reps, tune_cache, in_flight=1):
    """4 yr at dt = 2 s (63,115,200 samples, complex64), K = 300, 3843 modes, mixed: the whole
    step timed (also with `in_flight` waveforms in flight); mismatch of the full series against
    the FP64 GPU path."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300 import runtime as RT
    from paper_2104_04582_gb300 import tune
    w = W.config5()
    tr = RT.Trajectory(ctx, w.t_knots, w.modes)
    dev_in = tr.upload_inputs(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
    tr.set_data_device()
    out = RT.alloc_out(w.n_samples, True, dev.index)
    req = RT.request(tr, out, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_MIXED)
    slots = tr.info[2]
    tile, tuned_now = tune.ensure(ctx.handle, lambda: F.few_waveform(ctx.handle, req, sh),
                                  F.FEW_MIXED, slots, w.n_samples, tune_cache)

    def step():
        F.few_traj_set_data(ctx.handle, tr.handle, *dev_in, stream=sh)
        F.few_waveform(ctx.handle, req, sh)

    step()
    torch.cuda.synchronize()
    ms = _timed(stream, step, reps)  # the 505 MB output is larger than L2
    flight = None
    if in_flight > 1:
        sets = [(tr, dev_in, out, req)]
        for _ in range(in_flight - 1):
            t_ = RT.Trajectory(ctx, w.t_knots, w.modes)
            d_ = t_.upload_inputs(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
            o_ = RT.alloc_out(w.n_samples, True, dev.index)
            sets.append((t_, d_, o_, RT.request(t_, o_, w.n_samples, w.t0, w.dt, w.theta, w.phi,
                                                 F.FEW_MIXED)))
        streams = [torch.cuda.Stream(device=dev) for _ in sets]
        _in_flight(ctx, sets, streams, len(sets))  # warm-up
        n_steps = reps * len(sets)
        tot = _in_flight(ctx, sets, streams, n_steps)
        flight = {"in_flight": len(sets), "steps": n_steps, "ms_per_waveform": tot / n_steps,
                  "mode_samples_per_s": w.N * w.n_samples / (tot / n_steps * 1e-3),
                  "note": "each waveform its own trajectory and output, on its own stream"}
        for t_, _, _, _ in sets[1:]:
            t_.release()
        del sets
    out64 = RT.alloc_out(w.n_samples, False, dev.index)
    req64 = RT.request(tr, out64, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_FP64)
    F.few_waveform(ctx.handle, req64, sh)
    torch.cuda.synchronize()
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("device error in the stress run")
    a = out.to(torch.complex128)
    b = out64
    overlap = float(torch.sum(torch.conj(a) * b).real /
                    torch.sqrt(torch.sum(torch.abs(a) ** 2) * torch.sum(torch.abs(b) ** 2)))
    m = statistics.mean(ms)
    res = {"samples": w.n_samples, "knots": w.K, "modes": w.N, "slots": slots, "ms": m,
           "steps": reps, "mode_samples_per_s": w.N * w.n_samples / (m * 1e-3),
           "slot_samples_per_s": slots * w.n_samples / (m * 1e-3),
           "mismatch_vs_fp64_gpu_full_series": 1.0 - overlap, "tile": list(tile),
           "tile_tuned_in_this_run": tuned_now,
           "step": "spline build + harmonics + fold + phase anchors + mode sum, complex64 output"}
    if flight:
        res["in_flight"] = flight
    del a, out, out64
    tr.release()
    torch.cuda.synchronize()
    return res


def bench_serving_c4(ctx, n_req, budget_gb, tune_cache, loads=(0.5, 0.9, 1.2)):
    """Serving: a Poisson request stream from an MCMC-like client (0.5-4 yr, dt in {5,10,15} s,
    10-1000 modes, perturbed angles, phases and scale of resident trajectories, 10 % new ones),
    continuous batching with HBM-budget admission.  Every run starts with no trajectory on the
    device: the first request of each trajectory brings its knot data, and the server creates
    the trajectory and builds its splines on that request's path.  Capacity = completions/s of
    the whole stream submitted at once; then the stream at 50/90/120 % of that rate; the plain
    FP64 path's capacity on a tenth of the stream."""
    import dataclasses
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    from paper_2104_04582_gb300.serve import GpuEngine, Request, Server
    trajs_in, stream = W.config4_stream(n_req, rate_hz=1.0)
    slots_of = {k: F.few_mode_slots(w.modes)[0] for k, w in trajs_in.items()}

    def reqs_for(prec):
        out, seen = [], set()
        for r in stream:
            w = trajs_in[r.traj_key]
            first = r.traj_key not in seen
            seen.add(r.traj_key)
            out.append(Request(traj_key=r.traj_key, n_samples=w.n_samples, dt=w.dt, t0=w.t0,
                               theta=r.theta, phi=r.phi, scale=r.scale, dphi_phi0=r.dphi_phi0,
                               dphi_r0=r.dphi_r0, prec=prec, traj_inputs=w if first else None))
        return out

    mixed, plain_reqs = reqs_for(F.FEW_MIXED), reqs_for(F.FEW_FP64)
    work = lambda r: r.n_samples * slots_of[r.traj_key]
    tuner = GpuEngine(ctx)
    tiles = {}
    for reqs in (mixed, plain_reqs):
        med = sorted(reqs, key=work)[len(reqs) // 2]
        med = dataclasses.replace(med, traj_inputs=trajs_in[med.traj_key])
        tiles[med.prec] = tuner.tune_tiles(med, tune_cache)
    torch.cuda.synchronize()
    tuner.close()

    def run(reqs, rate_hz=None, seed=0):
        engine = GpuEngine(ctx)  # no trajectory resident: each is created by its first request
        srv = Server(engine, hbm_budget_bytes=int(budget_gb * 2 ** 30), max_batch=16,
                     max_inflight=3)
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
        torch.cuda.synchronize()
        engine.close()
        st["wall_s"] = wall
        st["offered_rate_hz"] = rate_hz
        return st

    run(mixed[:16])  # warm-up
    burst = run(mixed)
    cap = burst["completed"] / burst["wall_s"]
    res_loads = {}
    for f in loads:
        v = run(mixed, rate_hz=f * cap, seed=int(f * 100))
        res_loads[f"{int(round(f * 100))}%"] = {
            "offered_hz": v["offered_rate_hz"], "waveforms_per_s": v["waveforms_per_s"],
            "p50_ms": v["p50_ms"], "p99_ms": v["p99_ms"], "completed": v["completed"],
            "max_inflight_batches": v["max_inflight_batches"]}
    n_plain = max(8, n_req // 10)
    plain = run(plain_reqs[:n_plain])
    torch.cuda.synchronize()
    if ctx.sync_status() != F.FEW_OK:
        raise RuntimeError("device error in the serving run")
    samples = [trajs_in[r.traj_key].n_samples for r in stream]
    modes = [trajs_in[r.traj_key].N for r in stream]
    slot_samples = sum(slots_of[r.traj_key] * trajs_in[r.traj_key].n_samples for r in stream)
    res = {"requests": n_req, "trajectories": len(trajs_in),
           "trajectory_creation": "on the request path: the first request of each trajectory "
                                  "creates it and builds its splines from host knot data",
           "mean_samples": float(np.mean(samples)), "mean_modes": float(np.mean(modes)),
           "budget_gb": budget_gb, "max_batch": 16, "max_inflight": 3,
           "tiles": {("mixed" if p == F.FEW_MIXED else "fp64"): list(t) for p, t in tiles.items()},
           "capacity_mixed": {"value": cap, "unit": "waveforms/s", "p50_ms": burst["p50_ms"],
                              "p99_ms": burst["p99_ms"],
                              "c2_equivalent_waveforms_per_s_by_slot_samples":
                                  slot_samples / C2_SLOT_SAMPLES / burst["wall_s"]},
           "loads": res_loads,
           "plain_fp64_capacity": {"value": plain["completed"] / plain["wall_s"],
                                   "requests": plain["completed"], "p50_ms": plain["p50_ms"],
                                   "p99_ms": plain["p99_ms"]},
           "workload": "Poisson MCMC-like stream: 0.5-4 yr, dt in {5,10,15} s, 10-1000 modes, "
                       "perturbed angles/phases/scale of resident trajectories, 10% new ones "
                       "(created on their first request's path)",
           "seed": W.SEEDS["C4"]}
    res["capacity_vs_plain_fp64"] = cap / res["plain_fp64_capacity"]["value"]
    return res


def bench_selector(ctx, w, dev_in, dev, stream, sh):
    """Mode Selector (Sec. 3.D) on the benchmark's knot amplitudes, eps = 1e-5."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
    msk = torch.empty(w.N, dtype=torch.uint8, device=dev)
    mlist = np.ascontiguousarray(w.modes[:, 1])
    call = lambda: F.few_mode_select(ctx.handle, dev_in[2], dev_in[3], mlist, 1e-5, msk, sh)
    call()
    torch.cuda.synchronize()
    single = _timed(stream, call, 10)  # one call alone: includes the host's launch overhead
    n = 20
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n):  # back to back: each call's host work overlaps the previous kernel
        call()
    b.record(stream)
    torch.cuda.synchronize()
    return {"ms": a.elapsed_time(b) / n, "ms_single_call": statistics.mean(single),
            "timer": "CUDA events around 20 back-to-back calls (ms per call); ms_single_call "
                     "brackets one call alone, host launch work included",
            "eps": 1e-5, "knots": w.K, "modes": w.N, "selected": int(msk.sum().item()),
            "exact": "bit-exact against the oracle (tests)"}


def bench_direct(ctx, w, dev, stream, sh, nsd):
    """Direct (non-interpolated) summation over dense arrays, mixed: HBM-bound."""
    import torch
    from paper_2104_04582_gb300 import fewsum as F
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
    call = lambda: F.few_direct_sum(ctx.handle, d_pp, d_pr, d_re, d_im, w.modes, w.theta, w.phi,
                                    d_out, 1.0, F.FEW_MIXED, sh)
    call()
    torch.cuda.synchronize()
    msd = min(_timed(stream, call, 5))
    nbytes = nsd * (16 * w.N + 16 + 8)
    gbs = nbytes / (msd * 1e-3) / 1e9
    hbm = float(_peaks_file().get("hbm_gbs", 6800.0))
    return {"samples": nsd, "modes": w.N, "ms": msd,
            "mode_samples_per_s": nsd * w.N / (msd * 1e-3),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "bytes_per_launch": nbytes,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}}


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
    stream = torch.cuda.current_stream(dev)
    sh = int(stream.cuda_stream)
    prec = F.FEW_MIXED if args.prec == "mixed" else F.FEW_FP64
    flush = l2_flush_buffer(torch, dev)
    tune_cache = args.tune_cache or None

    r = bench_step_c2(args, ctx, w, dev, stream, sh, flush, prec, rank, world, tune_cache)
    out = dict(w=w, step_ms=r["step_ms"], seq_ms=r["seq_ms"], clocks=r["clocks"], h_fast=r["h"],
               slots=r["slots"],
               tile=r["tile"], tile_tuned_now=r["tile_tuned_now"], kernel_ms=r["kernel_ms"],
               sum_ms=r["sum_ms"], prec=prec, h_plain=None, plain=None, e2e=None, peaks={},
               timings_s={})
    if rank == 0:
        def timed_part(name, fn):
            t0 = time.perf_counter()
            v = fn()
            out["timings_s"][name] = round(time.perf_counter() - t0, 2)
            return v
        if not args.no_plain and prec == F.FEW_MIXED:
            out["plain"], out["h_plain"] = timed_part("plain_fp64", lambda: bench_plain_fp64(
                ctx, w, r["tr"], r["dev_in"], dev, stream, sh, flush, max(2, min(5, args.steps))))
        out["e2e"] = timed_part("e2e", lambda: bench_e2e(ctx, w, r["tr"], prec, sh, flush,
                                                         max(3, min(args.steps, 10)),
                                                         args.in_flight))
        out["selector"] = timed_part("mode_selector", lambda: bench_selector(
            ctx, w, r["dev_in"], dev, stream, sh))
        r["tr"].release()
        if args.batch > 0:
            out["batched_c3"] = timed_part("batched_c3", lambda: bench_batched_c3(
                ctx, dev, stream, sh, flush, args.batch, 3, tune_cache,
                in_flight=args.in_flight))
        if args.serving_requests > 0:
            out["serving"] = timed_part("serving", lambda: bench_serving_c4(
                ctx, args.serving_requests, args.serving_budget_gb, tune_cache))
        if not args.no_stress:
            out["stress_c5"] = timed_part("stress_c5", lambda: bench_stress_c5(
                ctx, dev, stream, sh, 3, tune_cache, in_flight=args.in_flight))
        if args.direct_samples > 0:
            out["direct"] = timed_part("direct_sum", lambda: bench_direct(
                ctx, w, dev, stream, sh, args.direct_samples))
        if args.rb_knots > 0:
            out["rb"] = timed_part("rb_amplitudes", lambda: bench_rb(ctx, args.rb_knots, w.N,
                                                                     stream, sh))
        if not args.no_probe:
            out["peaks"] = timed_part("pipe_probes", lambda: measure_peaks(local_rank))
        out["device_peaks"] = device_peaks(local_rank)
    else:
        r["tr"].release()
    torch.cuda.synchronize()
    ctx.close()
    return out


def assemble_line(args, res, ms, world):
    w = res["w"]
    fp32 = res["prec"] == 1
    slots = res["slots"]
    dp = res.get("device_peaks") or {}
    kms = statistics.mean(res["sum_ms"]) if res["sum_ms"] else float("nan")
    # algorithmic arithmetic of the summation kernel: one complex cubic (6 FMA) and one complex
    # Horner step (4 FMA) per (harmonic slot, sample); an FMA is 2 flops
    flops = 20.0 * slots * w.n_samples
    achieved = flops / (kms * 1e-3) / 1e12
    clocks = res["clocks"] or {}
    peak = dp.get("fp32_tflops" if fp32 else "fp64_tflops", float("nan"))
    traffic = None
    if (fp32 and PROFILED_TRAFFIC["bytes"] and
            _kernel_source_hash() == PROFILED_TRAFFIC["source_sha256_16"] and
            tuple(res.get("tile"))[:2] == PROFILED_TRAFFIC["tile"]):
        traffic = PROFILED_TRAFFIC["bytes"]
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
            "kernel": "k_sum<float,R> (mixed)" if fp32 else "k_sum<double,R> (fp64)",
            "kernel_ms": kms, "flops_per_launch": flops,
            "peak_source": ("nominal FP32 FMA: " if fp32 else "nominal FP64 FMA: ") +
                           dp.get("source", "") + " (ALU-bound kernel: neither HBM nor tensor peak applies)",
            "tile": list(res["tile"]), "tile_tuned_in_this_run": res["tile_tuned_now"]}
    probe = res["peaks"]
    if probe:
        key = "fp32_fma_per_s" if fp32 else "fp64_fma_per_s"
        if key in probe:
            pm = 2 * probe[key] / 1e12
            roof["peak_probe_tflops"] = pm
            roof["frac_of_probe"] = achieved / pm
        if fp32 and "fp32_fma_3reg_per_s" in probe:
            p3 = 2 * probe["fp32_fma_3reg_per_s"] / 1e12
            roof["peak_register_operand_tflops"] = p3
            roof["frac_of_register_operand_rate"] = achieved / p3
        if fp32 and "fp32_fma_summation_block_per_s" in probe:
            pb = 2 * probe["fp32_fma_summation_block_per_s"] / 1e12
            roof["peak_summation_block_tflops"] = pb
            roof["frac_of_summation_block_rate"] = achieved / pb
    if clocks.get("sm_mhz") and dp.get("sm_max_mhz"):
        roof["frac_at_measured_clock"] = achieved / (peak * clocks["sm_mhz"] / dp["sm_max_mhz"])
    value = aggregate_value(ms, world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
        "precision": ("mixed: FP64 phase splines and mod-2pi reduction (at anchors every 16 "
                      "samples, FP32 in-group increments); FP32 amplitudes, exponential powers "
                      "and accumulation") if fp32 else "fp64 throughout",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "seed": W.SEEDS["C2"], "knots": w.K, "modes": w.N,
                   "samples": w.n_samples, "harmonic_slots": slots,
                   "l2": ("not flushed: the steps rotate over %d sets of knot data, spline data "
                          "and output (~300 MB, more than L2)" % IN_FLIGHT_SETS
                          if args.in_flight > 1 else "flushed (256 MB write) between timed steps"),
                   "step": "spline build + harmonics + fold + phase anchors + mode sum, inputs "
                           "resident in HBM",
                   "in_flight": ("%d waveforms in flight on %d streams (independent waveforms "
                                 "overlap: the next one's kernels fill SMs the previous "
                                 "summation's CTAs have left)" % (args.in_flight, args.in_flight)
                                 if args.in_flight > 1 else "one waveform at a time"),
                   "parallelism": f"replicas x{world}"},
        "mode_samples_per_s": world * w.N * w.n_samples / (ms * 1e-3),
        "kernel_ms": res["kernel_ms"],
        "roofline": roof,
        "gpu_launches": (5 if fp32 else 4) * args.steps,
        "clocks": clocks or None,
        "e2e": res["e2e"],
    }
    seq = statistics.mean(res["seq_ms"])
    line["sequential"] = {"ms_per_step": seq, "value": aggregate_value(seq, world), "unit": UNIT,
                          "steps": args.steps,
                          "note": "one waveform at a time, L2 flushed before each step"}
    if res["plain"]:
        line["plain_fp64"] = res["plain"]
        line["speedup_vs_plain_fp64"] = res["plain"]["ms_per_step"] / seq  # both one at a time
    for key, name in (("batched_c3", "batched_c3"), ("serving", "serving"),
                      ("stress_c5", "stress_c5"), ("selector", "mode_selector"),
                      ("direct", "direct_sum"), ("rb", "rb_amplitudes")):
        if res.get(key):
            line[name] = res[key]
    if res["plain"]:
        pv = res["plain"]["value"]
        if res.get("batched_c3"):
            b = res["batched_c3"]
            b["c2_equivalent_vs_plain_fp64"] = b["c2_equivalent_waveforms_per_s_by_slot_samples"] / pv
        if res.get("serving"):
            s = res["serving"]
            s["c2_equivalent_vs_plain_fp64"] = (
                s["capacity_mixed"]["c2_equivalent_waveforms_per_s_by_slot_samples"] / pv)
    if res["peaks"]:
        line["measured_pipe_peaks"] = dict(res["peaks"])
    line["device_peaks"] = res.get("device_peaks")
    line["bench_sections_s"] = res["timings_s"]
    acc = {}
    if res["h_plain"] is not None:
        acc["mismatch_mixed_vs_fp64_full_series"] = _mismatch(res["h_fast"], res["h_plain"])
    if not args.no_cpu:
        cb, h_or = cpu_baseline(w, target_s=args.cpu_seconds)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        t_d = time.perf_counter()
        line["cpu_baseline_detail"] = cpu_baseline_detail(w)
        line["bench_sections_s"]["cpu_baseline_detail"] = round(time.perf_counter() - t_d, 2)
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
    return line


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


def reference_arm(args):
    """The oracle as it stands on the host cores, each step a bounded prefix of the workload."""
    w = W.config2()
    vals, step_s, cb = [], [], None
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb, _ = cpu_baseline(w, target_s=max(1.0, min(args.cpu_seconds, 60.0 / max(1, args.steps))))
        if k >= args.warmup:
            vals.append(cb["value"])
            step_s.append(time.perf_counter() - t0)
    v = statistics.median(vals)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(step_s), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "seed": W.SEEDS["C2"],
                       "note": "each step runs the oracle on a bounded prefix of the waveform "
                               "(ms_per_step is that step's measured wall time); value is the "
                               "whole-waveform rate extrapolated from the prefix"},
            "full_waveform_s_extrapolated": cb["seconds_full_waveform"],
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


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
    ap.add_argument("--no-stress", action="store_true", help="skip the 4-yr stress waveform")
    ap.add_argument("--in-flight", type=int, default=2,
                    help="waveforms in flight in the headline step (streams); 1 = one at a time "
                         "with the L2 flushed before each")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--rb-knots", type=int, default=6400,
                    help="knots of the reduced-basis amplitude measurement (0: skip)")
    ap.add_argument("--profile-case", choices=["mixed", "fp64", "direct", "rb", "select"],
                    default=None, help="untimed runs of the benchmark waveform for profiler captures")
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests of the serving measurement (0: skip)")
    ap.add_argument("--serving-budget-gb", type=float, default=16.0)
    ap.add_argument("--direct-samples", type=int, default=100000,
                    help="samples of the direct-summation measurement (0: skip)")
    ap.add_argument("--batch", type=int, default=256,
                    help="waveforms of the batched measurement (0: skip)")
    ap.add_argument("--tune-cache", default=os.path.join(ROOT, "build", "fewsum_tiles.json"),
                    help="tile cache of the autotuner ('' to tune without caching)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.profile_case:
        return run_profile_case(args.profile_case)

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args)))
        return 0

    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    res = run_gpu(args, rank, world, local_rank)
    ms = statistics.mean(res["step_ms"])
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
    print(json.dumps(assemble_line(args, res, ms, world)))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
