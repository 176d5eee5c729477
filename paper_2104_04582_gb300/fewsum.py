"""ctypes binding of libfewsum.so (include/fewsum.h), same names as the C ABI.

Argument marshalling only: every step of the waveform runs in the library's CUDA kernels.
PyTorch is used for device buffers and streams (``tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``); numpy arrays are passed as host pointers.
There is no CPU fallback: if the compiled library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import _build

FEW_OK = 0
FEW_ERR_INVALID_ARG = 1
FEW_ERR_KNOTS = 2
FEW_ERR_MODES = 3
FEW_ERR_RANGE = 4
FEW_ERR_NOMEM = 5
FEW_ERR_BUDGET = 6
FEW_ERR_CUDA = 7
FEW_ERR_TIMEOUT = 8
FEW_ERR_LIMIT = 9
FEW_ERR_STATE = 10

FEW_FP64 = 0
FEW_MIXED = 1
FEW_MEM_HOST = 0
FEW_MEM_DEVICE = 1
FEW_FRAME_SOURCE = 0
FEW_FRAME_SSB = 1
FEW_BATCH_REBUILD_SPLINES = 1
FEW_BATCH_NO_GRAPH = 2

# Every symbol include/fewsum.h declares (checked by the CPU test suite).
EXPORTED = [
    "few_strerror", "few_abi_version", "few_ctx_create", "few_ctx_destroy", "few_ctx_memory",
    "few_traj_create", "few_traj_set_data", "few_traj_release", "few_traj_info", "few_waveform",
    "few_batch_plan", "few_batch_run", "few_batch_release", "few_sync_status", "few_set_tiles",
    "few_get_tiles", "few_plan_segments", "few_mode_slots", "few_ctx_set_timing",
    "few_last_timing", "few_phase_samples", "few_waveform_noalloc",
    "few_mode_select", "few_direct_sum", "few_basis_create", "few_basis_release",
    "few_rb_amplitudes", "few_selftest_wait_expiry", "few_plan_cta_slices",
]


class few_request(ctypes.Structure):
    _fields_ = [
        ("traj", ctypes.c_void_p),
        ("theta", ctypes.c_double), ("phi", ctypes.c_double),
        ("scale", ctypes.c_double),
        ("dphi_phi0", ctypes.c_double), ("dphi_r0", ctypes.c_double),
        ("t0", ctypes.c_double), ("dt", ctypes.c_double),
        ("n_samples", ctypes.c_int64),
        ("prec", ctypes.c_int), ("out_c64", ctypes.c_int), ("out_where", ctypes.c_int),
        ("frame", ctypes.c_int),
        ("out", ctypes.c_void_p),
        ("theta_K", ctypes.c_double), ("phi_K", ctypes.c_double),
    ]


class FewError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = int(status)
        super().__init__(f"{fn}: {few_strerror(status)} ({status})")


_lib: Optional[ctypes.CDLL] = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)
_szp = ctypes.POINTER(ctypes.c_size_t)


def lib_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load the compiled library (no fallback: raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"libfewsum.so not found at {p}; build it with "
                               "paper_2104_04582_gb300._build.build()")
        L = ctypes.CDLL(p)
        sig = {
            "few_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "few_abi_version": (ctypes.c_int, []),
            "few_ctx_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t]),
            "few_ctx_destroy": (ctypes.c_int, [_vp]),
            "few_ctx_memory": (ctypes.c_int, [_vp, _szp, _szp]),
            "few_traj_create": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _ip, _ip, _ip, ctypes.c_int,
                                               ctypes.POINTER(_vp)]),
            "few_traj_set_data": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
            "few_traj_release": (ctypes.c_int, [_vp, _vp]),
            "few_traj_info": (ctypes.c_int, [_vp, _ip, _ip, _ip]),
            "few_waveform": (ctypes.c_int, [_vp, ctypes.POINTER(few_request), _vp]),
            "few_waveform_noalloc": (ctypes.c_int, [_vp, ctypes.POINTER(few_request), _vp]),
            "few_batch_plan": (ctypes.c_int, [_vp, ctypes.POINTER(few_request), ctypes.c_int,
                                              ctypes.c_uint, ctypes.POINTER(_vp)]),
            "few_batch_run": (ctypes.c_int, [_vp, _vp, _vp]),
            "few_batch_release": (ctypes.c_int, [_vp, _vp]),
            "few_sync_status": (ctypes.c_int, [_vp]),
            "few_set_tiles": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int]),
            "few_get_tiles": (ctypes.c_int, [_vp, ctypes.c_int, _ip, _ip, _ip]),
            "few_ctx_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
            "few_selftest_wait_expiry": (ctypes.c_int, [_vp, ctypes.c_uint, _vp]),
            "few_last_timing": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float)]),
            "few_phase_samples": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                                 _vp, _vp]),
            "few_mode_select": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _ip,
                                               ctypes.c_double, _vp, _vp]),
            "few_direct_sum": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, _ip, _ip, _ip,
                                              ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int, _vp, ctypes.c_int,
                                              _vp]),
            "few_basis_create": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
            "few_basis_release": (ctypes.c_int, [_vp, _vp]),
            "few_rb_amplitudes": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int,
                                                 _vp, _vp, _vp]),
            "few_plan_segments": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int64, _i64p]),
            "few_mode_slots": (ctypes.c_int, [_ip, _ip, _ip, ctypes.c_int, _ip, _ip]),
            "few_plan_cta_slices": (ctypes.c_int, [ctypes.c_int, _i64p, _ip, _ip, ctypes.c_int,
                                                   ctypes.c_int, _ip, _ip]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(fn: str, st: int) -> None:
    if st != FEW_OK:
        raise FewError(fn, st)


def few_strerror(status: int) -> str:
    return load().few_strerror(int(status)).decode()


def few_abi_version() -> int:
    return int(load().few_abi_version())


# ---------------------------------------------------------------- thin wrappers, same names

def few_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    h = _vp()
    _check("few_ctx_create", load().few_ctx_create(ctypes.byref(h), int(device), int(hbm_budget_bytes)))
    return h.value


def few_ctx_destroy(ctx: int) -> None:
    _check("few_ctx_destroy", load().few_ctx_destroy(ctx))


def few_ctx_memory(ctx: int):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check("few_ctx_memory", load().few_ctx_memory(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def few_traj_create(ctx: int, t_knots, modes) -> int:
    """modes: int array [N, 3] of (l, m >= 0, n)."""
    t = _f64(t_knots)
    md = _i32(modes).reshape(-1, 3)
    l, m, n = _i32(md[:, 0]), _i32(md[:, 1]), _i32(md[:, 2])
    h = _vp()
    st = load().few_traj_create(ctx, t.ctypes.data_as(_dp), len(t), l.ctypes.data_as(_ip),
                                m.ctypes.data_as(_ip), n.ctypes.data_as(_ip), len(l), ctypes.byref(h))
    _check("few_traj_create", st)
    return h.value


def few_traj_set_data(ctx: int, traj: int, phi_phi, phi_r, amp_re, amp_im, stream: int = 0) -> None:
    """Host numpy arrays (copied) or CUDA tensors (read in place on `stream`)."""
    arrs = (phi_phi, phi_r, amp_re, amp_im)
    if all(hasattr(a, "data_ptr") and getattr(a, "is_cuda", False) for a in arrs):
        for a in arrs:
            if not a.is_contiguous() or str(a.dtype) != "torch.float64":
                raise ValueError("device inputs must be contiguous float64 tensors")
        ptrs = [a.data_ptr() for a in arrs]
        where = FEW_MEM_DEVICE
        keep = arrs
    else:
        keep = [_f64(a) for a in arrs]
        ptrs = [a.ctypes.data for a in keep]
        where = FEW_MEM_HOST
    st = load().few_traj_set_data(ctx, traj, *ptrs, where, stream)
    del keep
    _check("few_traj_set_data", st)


def few_traj_release(ctx: int, traj: int) -> None:
    _check("few_traj_release", load().few_traj_release(ctx, traj))


def few_traj_info(traj: int):
    K, N, S = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("few_traj_info", load().few_traj_info(traj, ctypes.byref(K), ctypes.byref(N), ctypes.byref(S)))
    return K.value, N.value, S.value


def make_request(traj: int, out_ptr: int, n_samples: int, t0: float, dt: float, theta: float,
                 phi: float, scale: float = 1.0, prec: int = FEW_FP64, out_c64: bool = False,
                 out_where: int = FEW_MEM_DEVICE, dphi_phi0: float = 0.0,
                 dphi_r0: float = 0.0, frame: int = FEW_FRAME_SOURCE, theta_K: float = 0.0,
                 phi_K: float = 0.0) -> few_request:
    """theta, phi: source-frame angles, or the sky position when frame == FEW_FRAME_SSB."""
    return few_request(traj=traj, theta=float(theta), phi=float(phi), scale=float(scale),
                       dphi_phi0=float(dphi_phi0), dphi_r0=float(dphi_r0), t0=float(t0),
                       dt=float(dt), n_samples=int(n_samples), prec=int(prec),
                       out_c64=1 if out_c64 else 0, out_where=int(out_where), frame=int(frame),
                       out=out_ptr, theta_K=float(theta_K), phi_K=float(phi_K))


def few_waveform(ctx: int, req: few_request, stream: int = 0) -> None:
    _check("few_waveform", load().few_waveform(ctx, ctypes.byref(req), stream))


def few_waveform_noalloc(ctx: int, req: few_request, stream: int = 0) -> None:
    """few_waveform without any allocation (scratch in a fixed array inside the library).

    For callers that must not allocate once running; see include/fewsum.h for the size limit
    and the rule that overlapping calls must be ordered.
    """
    _check("few_waveform_noalloc", load().few_waveform_noalloc(ctx, ctypes.byref(req), stream))


def few_batch_plan(ctx: int, reqs: Sequence[few_request], flags: int = 0) -> int:
    arr = (few_request * len(reqs))(*reqs)
    h = _vp()
    _check("few_batch_plan", load().few_batch_plan(ctx, arr, len(reqs), int(flags), ctypes.byref(h)))
    return h.value


def few_batch_run(ctx: int, batch: int, stream: int = 0) -> None:
    _check("few_batch_run", load().few_batch_run(ctx, batch, stream))


def few_batch_release(ctx: int, batch: int) -> None:
    _check("few_batch_release", load().few_batch_release(ctx, batch))


def few_sync_status(ctx: int) -> int:
    """Returns the latched status code (does not raise)."""
    return int(load().few_sync_status(ctx))


def few_selftest_wait_expiry(ctx: int, limit_us: int, stream: int = 0) -> None:
    _check("few_selftest_wait_expiry", load().few_selftest_wait_expiry(ctx, int(limit_us), stream))


def few_set_tiles(ctx: int, prec: int, samples_per_thread: int, threads_per_block: int,
                  stage_slots: int) -> None:
    _check("few_set_tiles", load().few_set_tiles(ctx, int(prec), int(samples_per_thread),
                                                 int(threads_per_block), int(stage_slots)))


def few_get_tiles(ctx: int, prec: int):
    r, t, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("few_get_tiles", load().few_get_tiles(ctx, int(prec), ctypes.byref(r), ctypes.byref(t),
                                                 ctypes.byref(s)))
    return r.value, t.value, s.value


def few_ctx_set_timing(ctx: int, enable: bool) -> None:
    _check("few_ctx_set_timing", load().few_ctx_set_timing(ctx, 1 if enable else 0))


def few_last_timing(ctx: int):
    """[build, harmonics, fold, summation] ms of the most recent launches (-1: not recorded)."""
    ms = (ctypes.c_float * 4)()
    _check("few_last_timing", load().few_last_timing(ctx, ms))
    return [float(x) for x in ms]


def few_phase_samples(ctx: int, traj: int, t0: float, dt: float, n_samples: int, out_ptr: int,
                      dphi_phi0: float = 0.0, dphi_r0: float = 0.0, stream: int = 0) -> None:
    """Reduced orbital phases (turns) of every sample into a device buffer of 2*n doubles."""
    st = load().few_phase_samples(ctx, traj, float(t0), float(dt), int(n_samples),
                                  float(dphi_phi0), float(dphi_r0), out_ptr, stream)
    _check("few_phase_samples", st)


def few_mode_select(ctx: int, amp_re, amp_im, m, eps: float, mask, stream: int = 0) -> None:
    """Mode Selector on the device: amp_re/amp_im float64 CUDA tensors [K, N], m host ints [N],
    mask a uint8 CUDA tensor [N] (overwritten with the union of kept modes)."""
    K, N = int(amp_re.shape[0]), int(amp_re.shape[1])
    mm = _i32(m)
    st = load().few_mode_select(ctx, amp_re.data_ptr(), amp_im.data_ptr(), K, N,
                                mm.ctypes.data_as(_ip), float(eps), mask.data_ptr(), stream)
    _check("few_mode_select", st)


def few_direct_sum(ctx: int, phi_phi, phi_r, amp_re, amp_im, modes, theta: float, phi: float,
                   out, scale: float = 1.0, prec: int = FEW_MIXED, stream: int = 0) -> None:
    """Direct summation over dense device arrays (float64 CUDA tensors; amplitudes [Ns, N]) into
    a complex64/complex128 CUDA tensor `out` [Ns]."""
    md = _i32(modes).reshape(-1, 3)
    l, m, n = _i32(md[:, 0]), _i32(md[:, 1]), _i32(md[:, 2])
    c64 = str(out.dtype) == "torch.complex64"
    st = load().few_direct_sum(ctx, phi_phi.data_ptr(), phi_r.data_ptr(), amp_re.data_ptr(),
                               amp_im.data_ptr(), int(phi_phi.shape[0]), l.ctypes.data_as(_ip),
                               m.ctypes.data_as(_ip), n.ctypes.data_as(_ip), len(l), float(theta),
                               float(phi), float(scale), int(prec), out.data_ptr(),
                               1 if c64 else 0, stream)
    _check("few_direct_sum", st)


def few_basis_create(ctx: int, b_re, b_im, stream: int = 0) -> int:
    """Reduced basis [Nb, N] (real and imaginary parts) from host arrays (copied) or contiguous
    float64 CUDA tensors (read on `stream`)."""
    arrs = (b_re, b_im)
    if all(hasattr(a, "data_ptr") and getattr(a, "is_cuda", False) for a in arrs):
        for a in arrs:
            if not a.is_contiguous() or str(a.dtype) != "torch.float64":
                raise ValueError("device inputs must be contiguous float64 tensors")
        keep, ptrs, where = arrs, [a.data_ptr() for a in arrs], FEW_MEM_DEVICE
    else:
        keep = [_f64(a) for a in arrs]
        ptrs, where = [a.ctypes.data for a in keep], FEW_MEM_HOST
    if keep[0].shape != keep[1].shape or len(keep[0].shape) != 2:
        raise ValueError("basis parts must both be [Nb, N]")
    Nb, N = int(keep[0].shape[0]), int(keep[0].shape[1])
    h = _vp()
    st = load().few_basis_create(ctx, ptrs[0], ptrs[1], Nb, N, where, stream, ctypes.byref(h))
    del keep
    _check("few_basis_create", st)
    return h.value


def few_basis_release(ctx: int, basis: int) -> None:
    _check("few_basis_release", load().few_basis_release(ctx, basis))


def few_rb_amplitudes(ctx: int, basis: int, alpha_re, alpha_im, amp_re, amp_im, norms=None,
                      prec: int = FEW_MIXED, stream: int = 0) -> None:
    """Amplitudes [M, N] from reduced-basis coefficients [M, Nb] (float64 CUDA tensors), with
    optional target norms [M]; amp_re/amp_im are overwritten."""
    M = int(alpha_re.shape[0])
    st = load().few_rb_amplitudes(ctx, basis, alpha_re.data_ptr(), alpha_im.data_ptr(), M,
                                  None if norms is None else norms.data_ptr(), int(prec),
                                  amp_re.data_ptr(), amp_im.data_ptr(), stream)
    _check("few_rb_amplitudes", st)


def few_plan_segments(t_knots, t0: float, dt: float, n_samples: int) -> np.ndarray:
    t = _f64(t_knots)
    seg = np.zeros(len(t), dtype=np.int64)
    st = load().few_plan_segments(t.ctypes.data_as(_dp), len(t), float(t0), float(dt),
                                  int(n_samples), seg.ctypes.data_as(_i64p))
    _check("few_plan_segments", st)
    return seg


def few_plan_cta_slices(seg_starts, n_slots, grid: int, pass_samples: int):
    """CTA slices of the summation (host only): seg_starts a list of per-waveform segment start
    arrays (few_plan_segments), n_slots per waveform.  Returns (wave, sample) int arrays of
    length grid + 1."""
    segs = [np.ascontiguousarray(np.asarray(x, dtype=np.int64)) for x in seg_starts]
    cat = np.ascontiguousarray(np.concatenate(segs))
    K = _i32([len(x) for x in segs])
    sl = _i32(n_slots)
    wv = np.zeros(grid + 1, dtype=np.int32)
    sm = np.zeros(grid + 1, dtype=np.int32)
    _check("few_plan_cta_slices", load().few_plan_cta_slices(
        len(segs), cat.ctypes.data_as(_i64p), K.ctypes.data_as(_ip), sl.ctypes.data_as(_ip),
        int(grid), int(pass_samples), wv.ctypes.data_as(_ip), sm.ctypes.data_as(_ip)))
    return wv, sm


def few_mode_slots(modes):
    md = _i32(modes).reshape(-1, 3)
    l, m, n = _i32(md[:, 0]), _i32(md[:, 1]), _i32(md[:, 2])
    s, r = ctypes.c_int(), ctypes.c_int()
    st = load().few_mode_slots(l.ctypes.data_as(_ip), m.ctypes.data_as(_ip), n.ctypes.data_as(_ip),
                               len(l), ctypes.byref(s), ctypes.byref(r))
    _check("few_mode_slots", st)
    return s.value, r.value
