"""FP64 CPU oracle for the interpolated EMRI mode summation (arXiv:2104.04582).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package.  The product library
(``paper_2104_04582_gb300``) never imports, links or executes anything here, and this package
imports nothing from it: both sides consume the same seeded input arrays and nothing else.

The arithmetic lives in ``oracle.c`` (plain C, FP64, long double for the brute-force sum);
this module compiles it with gcc into ``oracle/_lib/liboracle.so`` on first use and wraps it
with numpy marshalling.  Function-by-function citations are in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB_PATH = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP, -O2, no target-specific flags).

    Expressions are evaluated as written (no contraction of a*b + c into a fused multiply-add,
    on x86-64 and on aarch64 alike), so every rounding step is the one the source shows.
    """
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(L: ctypes.CDLL) -> ctypes.CDLL:
    i64 = ctypes.c_int64
    L.oracle_spline_nak.argtypes = [_dp, ctypes.c_int, _dp, _dp]
    L.oracle_spline_nak.restype = ctypes.c_int
    L.oracle_spline_eval.argtypes = [_dp, ctypes.c_int, _dp, _dp, i64, _dp]
    L.oracle_spline_eval.restype = None
    L.oracle_swsh.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, _dp, _dp]
    L.oracle_swsh.restype = None
    wf = [_dp, ctypes.c_int, _dp, _dp, _ip, _ip, _ip, ctypes.c_int, _dp, _dp,
          ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
          ctypes.c_double]
    L.oracle_waveform.argtypes = wf + [i64, i64, _dp, ctypes.c_int]
    L.oracle_waveform.restype = ctypes.c_int
    L.oracle_direct_sum.argtypes = wf + [i64, _dp]
    L.oracle_direct_sum.restype = ctypes.c_int
    L.oracle_overlap.argtypes = [_dp, _dp, i64]
    L.oracle_overlap.restype = ctypes.c_double
    L.oracle_mismatch.argtypes = [_dp, _dp, i64]
    L.oracle_mismatch.restype = ctypes.c_double
    L.oracle_phases.argtypes = [_dp, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                i64, i64, _dp]
    L.oracle_phases.restype = ctypes.c_int
    L.oracle_mode_select.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_ubyte)]
    L.oracle_mode_select.restype = ctypes.c_int
    L.oracle_frame_angles.argtypes = [ctypes.c_double] * 4 + [_dp, _dp, _dp]
    L.oracle_frame_angles.restype = ctypes.c_int
    L.oracle_waveform_ssb.argtypes = [_dp, ctypes.c_int, _dp, _dp, _ip, _ip, _ip, ctypes.c_int, _dp,
                                      _dp] + [ctypes.c_double] * 7 + [i64, i64, _dp, ctypes.c_int]
    L.oracle_waveform_ssb.restype = ctypes.c_int
    L.oracle_direct_dense.argtypes = [_dp, _dp, i64, _ip, _ip, _ip, ctypes.c_int, _dp, _dp,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp,
                                       ctypes.c_int]
    L.oracle_direct_dense.restype = ctypes.c_int
    L.oracle_rb_amplitudes.argtypes = [ctypes.c_int] * 3 + [_dp] * 5 + [_dp, _dp, ctypes.c_int]
    L.oracle_rb_amplitudes.restype = ctypes.c_int
    L.oracle_max_threads.argtypes = []
    L.oracle_max_threads.restype = ctypes.c_int
    return L


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Temporarily route every wrapper in this module to another compiled oracle.

    Used only by the mutation tests, which compile deliberately broken copies of oracle.c
    to show that the pins reject them.
    """

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self._saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray):
    return a.ctypes.data_as(_dp)


class OracleError(RuntimeError):
    pass


def spline_nak(t, y) -> np.ndarray:
    """Not-a-knot cubic spline coefficients [K-1, 4] in local x = t - t_k (Sec. 3.C)."""
    t, y = _d(t), _d(y)
    coef = np.zeros((len(t) - 1, 4)) if len(t) > 1 else np.zeros((0, 4))
    rc = lib().oracle_spline_nak(_p(t), len(t), _p(y), _p(coef))
    if rc:
        raise OracleError(f"oracle_spline_nak: status {rc}")
    return coef


def spline_eval(t, coef, x) -> np.ndarray:
    t, coef, x = _d(t), _d(coef), _d(x)
    out = np.zeros(len(x))
    lib().oracle_spline_eval(_p(t), len(t), _p(coef), _p(x), len(x), _p(out))
    return out


def swsh(s: int, l: int, m: int, theta: float, phi: float) -> complex:
    """Spin-weighted spherical harmonic sY_lm(theta, phi) (Wigner-d explicit sum)."""
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().oracle_swsh(int(s), int(l), int(m), float(theta), float(phi), ctypes.byref(re),
                      ctypes.byref(im))
    return complex(re.value, im.value)


def _modes(modes):
    modes = np.ascontiguousarray(modes, dtype=np.int32).reshape(-1, 3)
    l = np.ascontiguousarray(modes[:, 0])
    m = np.ascontiguousarray(modes[:, 1])
    n = np.ascontiguousarray(modes[:, 2])
    return l, m, n


def _wave_args(t, phi_phi, phi_r, modes, amp_re, amp_im):
    t, pp, pr = _d(t), _d(phi_phi), _d(phi_r)
    l, m, n = _modes(modes)
    ar, ai = _d(amp_re), _d(amp_im)
    N = len(l)
    if ar.shape != (len(t), N) or ai.shape != (len(t), N):
        raise ValueError("amplitudes must be [K, N]")
    keep = (t, pp, pr, l, m, n, ar, ai)
    ip = lambda a: a.ctypes.data_as(_ip)
    args = [_p(t), len(t), _p(pp), _p(pr), ip(l), ip(m), ip(n), N, _p(ar), _p(ai)]
    return keep, args


def waveform(t, phi_phi, phi_r, modes, amp_re, amp_im, theta, phi, scale=1.0, t0=0.0,
             dt=10.0, i_begin=0, count=0, nthreads=1) -> np.ndarray:
    """h(t_i) for t_i = t0 + i*dt, i in [i_begin, i_begin+count): complex128 array."""
    keep, args = _wave_args(t, phi_phi, phi_r, modes, amp_re, amp_im)
    out = np.zeros(2 * int(count))
    rc = lib().oracle_waveform(*args, float(theta), float(phi), float(scale), float(t0),
                               float(dt), int(i_begin), int(count), _p(out), int(nthreads))
    if rc:
        raise OracleError(f"oracle_waveform: status {rc}")
    del keep
    return out.view(np.complex128)


def direct_sum(t, phi_phi, phi_r, modes, amp_re, amp_im, theta, phi, scale=1.0, t0=0.0,
               dt=10.0, count=0) -> np.ndarray:
    """Brute-force signed-list sum in long double with unreduced phases (tiny inputs)."""
    keep, args = _wave_args(t, phi_phi, phi_r, modes, amp_re, amp_im)
    out = np.zeros(2 * int(count))
    rc = lib().oracle_direct_sum(*args, float(theta), float(phi), float(scale), float(t0),
                                 float(dt), int(count), _p(out))
    if rc:
        raise OracleError(f"oracle_direct_sum: status {rc}")
    del keep
    return out.view(np.complex128)


def phases(t, phi_phi, phi_r, t0, dt, i_begin, count) -> np.ndarray:
    """Orbital phases at the samples, each reduced mod 2 pi, in turns: float64 [count, 2]."""
    t, pp, pr = _d(t), _d(phi_phi), _d(phi_r)
    out = np.zeros(2 * int(count))
    rc = lib().oracle_phases(_p(t), len(t), _p(pp), _p(pr), float(t0), float(dt), int(i_begin),
                             int(count), _p(out))
    if rc:
        raise OracleError(f"oracle_phases: status {rc}")
    return out.reshape(-1, 2)


def mode_select(amp_re, amp_im, modes, eps) -> np.ndarray:
    """Mode Selector (Sec. 3.D): boolean mask [N] of the modes kept at some knot."""
    ar, ai = _d(amp_re), _d(amp_im)
    K, N = ar.shape
    m = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, 3)[:, 1])
    mask = np.zeros(N, dtype=np.uint8)
    lib().oracle_mode_select(_p(ar), _p(ai), K, N, m.ctypes.data_as(_ip), float(eps),
                             mask.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return mask.astype(bool)


def frame_angles(theta_S, phi_S, theta_K, phi_K):
    """(theta_src, phi_src, psi) of the frame transformation (Sec. 2.A)."""
    th, ph, psi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib().oracle_frame_angles(float(theta_S), float(phi_S), float(theta_K), float(phi_K),
                                   ctypes.byref(th), ctypes.byref(ph), ctypes.byref(psi))
    if rc:
        raise OracleError(f"oracle_frame_angles: status {rc}")
    return th.value, ph.value, psi.value


def waveform_ssb(t, phi_phi, phi_r, modes, amp_re, amp_im, theta_S, phi_S, theta_K, phi_K,
                 scale=1.0, t0=0.0, dt=10.0, i_begin=0, count=0, nthreads=1) -> np.ndarray:
    """Detector-frame waveform: source-frame sum at the transformed angles, times -e^{-2i psi}."""
    keep, args = _wave_args(t, phi_phi, phi_r, modes, amp_re, amp_im)
    out = np.zeros(2 * int(count))
    rc = lib().oracle_waveform_ssb(*args, float(theta_S), float(phi_S), float(theta_K),
                                   float(phi_K), float(scale), float(t0), float(dt), int(i_begin),
                                   int(count), _p(out), int(nthreads))
    if rc:
        raise OracleError(f"oracle_waveform_ssb: status {rc}")
    del keep
    return out.view(np.complex128)


def direct_dense(phi_phi, phi_r, modes, amp_re, amp_im, theta, phi, scale=1.0,
                 nthreads=1) -> np.ndarray:
    """Direct summation over arrays given at every sample (Sec. 3.C): complex128 [n_samples]."""
    pp, pr = _d(phi_phi), _d(phi_r)
    l, m, n = _modes(modes)
    ar, ai = _d(amp_re), _d(amp_im)
    ns = len(pp)
    if ar.shape != (ns, len(l)) or ai.shape != (ns, len(l)) or len(pr) != ns:
        raise ValueError("amplitudes must be [n_samples, N]")
    out = np.zeros(2 * ns)
    ip = lambda a: a.ctypes.data_as(_ip)
    rc = lib().oracle_direct_dense(_p(pp), _p(pr), ns, ip(l), ip(m), ip(n), len(l), _p(ar), _p(ai),
                                   float(theta), float(phi), float(scale), _p(out), int(nthreads))
    if rc:
        raise OracleError(f"oracle_direct_dense: status {rc}")
    return out.view(np.complex128)


def rb_amplitudes(alpha, basis, norms=None, nthreads=1) -> np.ndarray:
    """Reduced-basis amplitudes (Sec. 3.E): alpha [M, Nb] complex, basis [Nb, N] complex,
    optional target norms [M]; returns complex128 [M, N]."""
    a = np.ascontiguousarray(alpha, dtype=np.complex128)
    b = np.ascontiguousarray(basis, dtype=np.complex128)
    if a.ndim != 2 or b.ndim != 2 or a.shape[1] != b.shape[0]:
        raise ValueError("alpha must be [M, Nb] and basis [Nb, N]")
    M, Nb = a.shape
    N = b.shape[1]
    ar, ai = _d(a.real), _d(a.imag)
    br, bi = _d(b.real), _d(b.imag)
    nu = None if norms is None else _d(norms)
    if nu is not None and nu.shape != (M,):
        raise ValueError("norms must be [M]")
    out_re, out_im = np.zeros((M, N)), np.zeros((M, N))
    rc = lib().oracle_rb_amplitudes(M, Nb, N, _p(ar), _p(ai), _p(br), _p(bi),
                                    None if nu is None else _p(nu), _p(out_re), _p(out_im),
                                    int(nthreads))
    if rc:
        raise OracleError(f"oracle_rb_amplitudes: status {rc}")
    return out_re + 1j * out_im


def _c(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


def overlap(a, b) -> float:
    """<a|b>/sqrt(<a|a><b|b>) with S_n = 1 (Sec. 6), time-domain form."""
    x, y = _c(a), _c(b)
    return float(lib().oracle_overlap(_p(x), _p(y), len(x) // 2))


def mismatch(a, b) -> float:
    """1 - overlap(a, b), evaluated as 0.5*||a/|a| - b/|b|||^2."""
    x, y = _c(a), _c(b)
    return float(lib().oracle_mismatch(_p(x), _p(y), len(x) // 2))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def waveform_inputs(w, i_begin=0, count=None, nthreads=1, scale=None) -> np.ndarray:
    """Convenience: oracle waveform for a ``workloads.WaveformInputs``-like object."""
    if count is None:
        count = w.n_samples - i_begin
    return waveform(w.t_knots, w.phi_phi, w.phi_r, w.modes, w.amp_re, w.amp_im, w.theta, w.phi,
                    w.scale if scale is None else scale, w.t0, w.dt, i_begin, count, nthreads)
