"""Planted mistakes in the oracle must be caught by its pins.

Each case compiles a copy of oracle.c with one plausible mistake (a dropped term, a wrong sign,
a transposed operand, a wrong index) into a temporary library, routes the oracle wrappers to
it, and checks that at least one independent pin (closed form, library cross-check, brute
force) now fails.  Everything runs on the CPU.
"""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTATIONS = {
    "partner_sign_dropped": ("double sg = (l[i] & 1) ? -1.0 : 1.0;", "double sg = 1.0;"),
    "partner_for_m0": [("if (m[i] > 0) {\n            double a, b;",
                        "if (m[i] >= 0) {\n            double a, b;"),
                       ("if (m[i] > 0) {\n                /* conj(A) Y- (c + i s) */",
                        "if (m[i] >= 0) {\n                /* conj(A) Y- (c + i s) */")],
    "partner_uses_plus_m": ("oracle_swsh(-2, l[i], -m[i], theta, phi, &a, &b);\n            double sg",
                            "oracle_swsh(-2, l[i], m[i], theta, phi, &a, &b);\n            double sg"),
    "exponent_sign": ("hr += ayr * c + ayi * s;", "hr += ayr * c - ayi * s;"),
    "m_n_transposed": ("double ph = (double)m[i] * fphi + (double)n[i] * fr;",
                       "double ph = (double)n[i] * fphi + (double)m[i] * fr;"),
    "nak_row0_coeff": ("b[0] = ((2.0 * h[1] + 3.0 * h[0])", "b[0] = ((2.0 * h[1] + 2.0 * h[0])"),
    "nak_last_row_index": ("dl[n - 2] = a + c;", "dl[n - 2] = a + a;"),
    "pivot_rhs_sign": ("b[k + 1] = bk - mult * b[k];", "b[k + 1] = bk + mult * b[k];"),
    "c3_coefficient": ("(s[k] + s[k + 1] - 2.0 * d[k]) / (h[k] * h[k])",
                       "(s[k] + s[k + 1] - 2.0 * d[k]) / (h[k])"),
    "wigner_power": ("powl(c, (long double)(2 * j + m - mp - 2 * k))",
                     "powl(c, (long double)(2 * j - m + mp - 2 * k))"),
    "ylm_norm": ("(2.0L * l + 1.0L) / (4.0L *", "(2.0L * l + 3.0L) / (4.0L *"),
    "scale_dropped": ("out[2 * j] = scale * hr;", "out[2 * j] = hr;"),
    "select_no_doubling": ("if (m[i] > 0) p *= 2.0;", ""),
    "direct_partner_sign": ("double byr = Ar * ymr[i] + Ai * ymi[i], byi = Ar * ymi[i] - Ai * ymr[i];",
                            "double byr = Ar * ymr[i] - Ai * ymi[i], byi = Ar * ymi[i] + Ai * ymr[i];"),
    "frame_psi_sign": ("double num = cos(tS) * sin(tK) * cos(pS - pK) - sin(tS) * cos(tK);",
                       "double num = cos(tS) * sin(tK) * cos(pS - pK) + sin(tS) * cos(tK);"),
    "frame_no_pi_shift": ("double fr = -cos(2.0 * psi), fi = sin(2.0 * psi);",
                          "double fr = cos(2.0 * psi), fi = -sin(2.0 * psi);"),
    "rb_cross_term_sign": ("si += ar * bi + ai * br;", "si += ar * bi - ai * br;"),
    "rb_conjugated_basis": ("sr += ar * br - ai * bi;", "sr += ar * br + ai * bi;"),
    "rb_norm_not_rooted": ("(long double)norms[k] / sqrtl(nn)", "(long double)norms[k] / nn"),
    "rb_basis_row_fixed": ("b_re[(size_t)j * N + i], bi = b_im[(size_t)j * N + i];",
                           "b_re[(size_t)i], bi = b_im[(size_t)i];"),
    "select_drops_boundary_mode": [("            mask[e[j].i] = 1;\n            if (c >= target) break;",
                                    "            if (c >= target) break;\n            mask[e[j].i] = 1;")],
}


def _m2y2(m, th, ph):
    c, s = math.cos(th), math.sin(th)
    amp = {2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
           1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c),
           0: math.sqrt(15 / (32 * math.pi)) * s * s,
           -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
           -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2}[m]
    return amp * complex(math.cos(m * ph), math.sin(m * ph))


def _pins_hold() -> bool:
    """A compact run of the independent pins; False as soon as one fails."""
    interp = pytest.importorskip("scipy.interpolate")
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(0)
    # spline vs scipy, on smooth and on strongly non-uniform knots (exercises pivoting)
    for t in (W.knot_times(1e6, 30),
              np.cumsum(np.r_[0.0, 1.0, 1.0, 80.0, 0.5, 0.5, 90.0, 1.0, 60.0, 1.0])):
        y = rng.normal(size=len(t))
        coef = oracle.spline_nak(t, y)
        ref = interp.CubicSpline(t, y, bc_type="not-a-knot").c[::-1].T
        if np.max(np.abs(coef - ref)) > 1e-9 * np.max(np.abs(ref)):
            return False
    # harmonics: l = 2 closed forms and spin-0 against scipy
    for m in range(-2, 3):
        if abs(oracle.swsh(-2, 2, m, 1.2, 0.4) - _m2y2(m, 1.2, 0.4)) > 1e-14:
            return False
    f = getattr(sp, "sph_harm_y", None)
    for l in (3, 6):
        for m in (-2, 1, 3):
            ref = complex(f(l, m, 0.8, 2.0)) if f else complex(sp.sph_harm(m, l, 2.0, 0.8))
            if abs(oracle.swsh(0, l, m, 0.8, 2.0) - ref) > 1e-13:
                return False
    for l in (4, 7):
        tot = sum(abs(oracle.swsh(-2, l, m, 0.7, 0.1)) ** 2 for m in range(-l, l + 1))
        if abs(tot - (2 * l + 1) / (4 * math.pi)) > 1e-13:
            return False
    # single-mode closed forms (l = 2 and m = 0, Y from the textbook forms)
    T, K, dt = 2.0e5, 9, 37.0
    t = W.knot_times(T, K)
    for (l, m, n) in ((2, 2, 3), (2, 1, -1), (2, 0, 2)):
        A = 0.7 - 0.3j
        pphi, pr = 2.1e-3 * t + 0.4, 1.7e-3 * t + 2.9
        ns = int(T / dt)
        h = oracle.waveform(t, pphi, pr, [(l, m, n)], np.full((K, 1), A.real),
                            np.full((K, 1), A.imag), 1.1, 0.6, 1.7, 0.0, dt, 0, ns)
        ts = np.arange(ns) * dt
        Phi = m * (2.1e-3 * ts + 0.4) + n * (1.7e-3 * ts + 2.9)
        want = A * _m2y2(m, 1.1, 0.6) * np.exp(-1j * Phi)
        if m > 0:
            want = want + np.conj(A) * _m2y2(-m, 1.1, 0.6) * np.exp(1j * Phi)
        want *= 1.7
        if np.max(np.abs(h - want)) > 1e-12 * np.max(np.abs(want)):
            return False
    # mode selector: geometric closed form and the m > 0 doubling
    r, N, eps = 0.8, 60, 1e-5
    pg = r ** np.arange(N)
    mg = np.stack([np.full(N, 2), np.zeros(N, int), np.arange(N)], axis=1)
    kept = oracle.mode_select(np.sqrt(pg)[None, :], np.zeros((1, N)), mg, eps)
    if kept.sum() != math.ceil(math.log(eps + (1 - eps) * r ** N) / math.log(r)):
        return False
    md = np.stack([np.full(6, 2), np.array([0, 0, 0, 1, 0, 0]), np.arange(6)], axis=1)
    re2 = np.array([[1.0, 0.5, 0.0, 0.5, 0.0, 0.0]])
    if list(oracle.mode_select(re2, np.zeros_like(re2), md, 0.3)) != [True, False, False, True,
                                                                        False, False]:
        return False
    # frame transformation: psi against the vector form, and the detector-frame composition
    R = np.array([math.sin(0.54) * math.cos(5.36), math.sin(0.54) * math.sin(5.36), math.cos(0.54)])
    S = np.array([math.sin(1.73) * math.cos(3.2), math.sin(1.73) * math.sin(3.2), math.cos(1.73)])
    z = np.array([0.0, 0.0, 1.0])
    th, ph, psi = oracle.frame_angles(0.54, 5.36, 1.73, 3.2)
    want = math.atan2(S @ z - (S @ R) * (z @ R), R @ np.cross(S, z))
    if abs(np.exp(2j * psi) - np.exp(2j * want)) > 1e-12:
        return False
    wt = W.tiny_inputs(5, n_samples=50)
    src = oracle.waveform(wt.t_knots, wt.phi_phi, wt.phi_r, wt.modes, wt.amp_re, wt.amp_im, th,
                          ph, 1.0, wt.t0, wt.dt, 0, 50)
    ssb = oracle.waveform_ssb(wt.t_knots, wt.phi_phi, wt.phi_r, wt.modes, wt.amp_re, wt.amp_im,
                              0.54, 5.36, 1.73, 3.2, 1.0, wt.t0, wt.dt, 0, 50)
    if np.max(np.abs(ssb + np.exp(-2j * psi) * src)) > 1e-13 * np.max(np.abs(src)):
        return False
    # direct summation: single-mode closed form
    ts = np.arange(500) * 17.0
    A = 0.3 + 0.8j
    hd = oracle.direct_dense(2.1e-3 * ts + 0.4, 1.7e-3 * ts + 2.9, [(2, 1, -2)],
                             np.full((500, 1), A.real), np.full((500, 1), A.imag), 0.9, 2.2)
    Phi = 1 * (2.1e-3 * ts + 0.4) - 2 * (1.7e-3 * ts + 2.9)
    wd = A * _m2y2(1, 0.9, 2.2) * np.exp(-1j * Phi) + np.conj(A) * _m2y2(-1, 0.9, 2.2) * np.exp(1j * Phi)
    if np.max(np.abs(hd - wd)) > 1e-12 * np.max(np.abs(wd)):
        return False
    # reduced-basis amplitudes: the hand-worked product, its renormalisation, the Fourier basis
    ab = np.array([[1 + 2j, 3 - 1j]])
    Bh = np.array([[1, 1j, 0], [2, 0, -1]], dtype=complex)
    if not np.array_equal(oracle.rb_amplitudes(ab, Bh), np.array([[7, -2 + 1j, -3 + 1j]])):
        return False
    if not np.array_equal(oracle.rb_amplitudes(ab, Bh, norms=[2.0]),
                          np.array([[1.75, -0.5 + 0.25j, -0.75 + 0.25j]])):
        return False
    jj, ii = np.meshgrid(np.arange(5), np.arange(16), indexing="ij")
    af = rng.normal(size=(2, 5)) + 1j * rng.normal(size=(2, 5))
    if np.max(np.abs(oracle.rb_amplitudes(af, np.exp(-2j * np.pi * jj * ii / 16))
                     - np.fft.fft(af, n=16, axis=1))) > 1e-12:
        return False
    # shortcut vs brute force on odd and even l
    w = W.tiny_inputs(3, K=8, n_samples=200)
    a = oracle.waveform_inputs(w)
    b = oracle.direct_sum(w.t_knots, w.phi_phi, w.phi_r, w.modes, w.amp_re, w.amp_im, w.theta,
                          w.phi, 1.0, w.t0, w.dt, w.n_samples)
    if np.linalg.norm(a - b) > 1e-12 * np.linalg.norm(b):
        return False
    return True


def _build_variant(tmp_path, name, edits):
    src = open(SRC).read()
    if isinstance(edits, tuple):
        edits = [edits]
    for old, new in edits:
        # a mistake in a line that occurs in several routines is planted in every copy
        assert src.count(old) >= 1, f"mutation anchor not found: {name}"
        src = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-std=c11", "-shared", "-fPIC", str(path), "-o",
                    str(so), "-lm"], check=True)
    return str(so)


def test_unmutated_oracle_passes_the_compact_pins():
    assert _pins_hold()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    so = _build_variant(tmp_path, name, MUTATIONS[name])
    with oracle.use_library(so):
        assert not _pins_hold(), f"planted mistake {name!r} was not caught"
