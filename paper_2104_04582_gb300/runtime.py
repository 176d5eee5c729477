"""Owning wrappers around the C ABI handles, with torch device buffers and streams.

These classes only marshal arguments (numpy/torch -> pointers) and manage handle lifetimes;
the waveform itself is computed by libfewsum.so.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import fewsum as F


def _torch():
    import torch  # deferred: the package is importable without torch on CPU-only tools
    return torch


class Context:
    """A few_ctx on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.handle = F.few_ctx_create(device, hbm_budget_bytes)

    def close(self) -> None:
        if self.handle:
            F.few_ctx_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync_status(self) -> int:
        return F.few_sync_status(self.handle)

    def set_tiles(self, prec: int, samples_per_thread: int, threads: int,
                  stage_slots: Optional[int] = None) -> None:
        """Tile shape of one precision; stage_slots (the mode tile) keeps its value if None."""
        if stage_slots is None:
            stage_slots = F.few_get_tiles(self.handle, prec)[2]
        F.few_set_tiles(self.handle, prec, samples_per_thread, threads, stage_slots)

    def get_tiles(self, prec: int):
        """(samples per thread, threads per block, slots per stage) of one precision."""
        return F.few_get_tiles(self.handle, prec)

    def memory(self):
        return F.few_ctx_memory(self.handle)


def current_stream() -> int:
    return int(_torch().cuda.current_stream().cuda_stream)


class Trajectory:
    """A few_traj: knot grid + mode list; spline data set from host or device arrays."""

    def __init__(self, ctx: Context, t_knots, modes):
        self.ctx = ctx
        self.t_knots = np.ascontiguousarray(t_knots, dtype=np.float64)
        self.modes = np.ascontiguousarray(modes, dtype=np.int32).reshape(-1, 3)
        self.handle = F.few_traj_create(ctx.handle, self.t_knots, self.modes)
        self._dev_inputs = None

    @property
    def info(self):
        return F.few_traj_info(self.handle)

    def set_data_host(self, phi_phi, phi_r, amp_re, amp_im, stream: Optional[int] = None) -> None:
        F.few_traj_set_data(self.ctx.handle, self.handle, phi_phi, phi_r, amp_re, amp_im,
                            current_stream() if stream is None else stream)

    def upload_inputs(self, phi_phi, phi_r, amp_re, amp_im):
        """Copy knot data to device tensors (kept alive by this object) and return them."""
        torch = _torch()
        dev = torch.device("cuda", self.ctx.device)
        self._dev_inputs = tuple(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).to(dev)
                                 for a in (phi_phi, phi_r, amp_re, amp_im))
        return self._dev_inputs

    def set_data_device(self, tensors=None, stream: Optional[int] = None) -> None:
        t = tensors if tensors is not None else self._dev_inputs
        F.few_traj_set_data(self.ctx.handle, self.handle, *t,
                            stream=current_stream() if stream is None else stream)

    def release(self) -> None:
        if self.handle:
            F.few_traj_release(self.ctx.handle, self.handle)
            self.handle = 0


def from_inputs(ctx: Context, w, device_data: bool = True) -> Trajectory:
    """Trajectory for a workloads.WaveformInputs, spline data set from device (default) or host."""
    tr = Trajectory(ctx, w.t_knots, w.modes)
    if device_data:
        tr.upload_inputs(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
        tr.set_data_device()
    else:
        tr.set_data_host(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
    return tr


def alloc_out(n_samples: int, c64: bool, device: int = 0):
    torch = _torch()
    return torch.empty(int(n_samples), dtype=torch.complex64 if c64 else torch.complex128,
                       device=torch.device("cuda", device))


def request(tr: Trajectory, out, n_samples: int, t0: float, dt: float, theta: float, phi: float,
            prec: int = F.FEW_FP64, scale: float = 1.0, dphi_phi0: float = 0.0,
            dphi_r0: float = 0.0, out_where: int = F.FEW_MEM_DEVICE, frame: int = F.FEW_FRAME_SOURCE,
            theta_K: float = 0.0, phi_K: float = 0.0) -> F.few_request:
    if out_where == F.FEW_MEM_DEVICE:
        ptr = out.data_ptr()
        c64 = str(out.dtype) == "torch.complex64"
    else:
        ptr = out.ctypes.data
        c64 = out.dtype == np.complex64
    return F.make_request(tr.handle, ptr, n_samples, t0, dt, theta, phi, scale, prec, c64,
                          out_where, dphi_phi0, dphi_r0, frame, theta_K, phi_K)


def waveform(ctx: Context, tr: Trajectory, n_samples: int, t0: float, dt: float, theta: float,
             phi: float, prec: int = F.FEW_FP64, c64: Optional[bool] = None, scale: float = 1.0,
             dphi_phi0: float = 0.0, dphi_r0: float = 0.0, stream: Optional[int] = None, out=None):
    """Queue one waveform into a (new or given) device tensor and return the tensor."""
    if c64 is None:
        c64 = prec == F.FEW_MIXED
    if out is None:
        out = alloc_out(n_samples, c64, ctx.device)
    req = request(tr, out, n_samples, t0, dt, theta, phi, prec, scale, dphi_phi0, dphi_r0)
    F.few_waveform(ctx.handle, req, current_stream() if stream is None else stream)
    return out


def waveform_inputs(ctx: Context, tr: Trajectory, w, prec: int = F.FEW_FP64, c64=None,
                    i_begin: int = 0, count: Optional[int] = None, **kw):
    """Waveform of a workloads.WaveformInputs, optionally a sample window [i_begin, +count)."""
    if count is None:
        count = w.n_samples - i_begin
    return waveform(ctx, tr, count, w.t0 + i_begin * w.dt, w.dt, w.theta, w.phi, prec, c64,
                    w.scale, **kw)
