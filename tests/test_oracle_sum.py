"""Pins for the oracle's interpolated mode sum (Sec. 4 sum, Eq. amp_symmetry) and mismatch.

* single-mode closed form: constant amplitude and phases linear in t make every spline exact,
  so h(t) = scale*[A Y+ e^{-i Phi} + (-1)^l conj(A) -2Y_{l,-m} e^{+i Phi}] analytically, with
  Y from the textbook l = 2 forms (independent of the oracle's harmonics);
* symmetry: the folded m >= 0 sum equals the brute-force signed-list sum (long double,
  unreduced phases) on tiny inputs;
* linearity in the amplitudes and in the scale;
* the mismatch definition (Sec. 6) on cases with known values;
* mode counts printed in the paper (tests/golden/mode_counts.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _m2y2(m, th, ph):
    c, s = math.cos(th), math.sin(th)
    amp = {2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
           1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c),
           0: math.sqrt(15 / (32 * math.pi)) * s * s,
           -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
           -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2}[m]
    return amp * complex(math.cos(m * ph), math.sin(m * ph))


def _linear_traj(K, T, wphi, wr, c_phi, c_r):
    t = W.knot_times(T, K)
    return t, wphi * t + c_phi, wr * t + c_r


@pytest.mark.parametrize("mode", [(2, 2, 0), (2, 2, 3), (2, 1, -4), (2, 0, 5), (2, 0, -2)])
def test_single_mode_closed_form_l2(mode):
    l, m, n = mode
    T, K, dt = 2.0e5, 9, 37.0
    wphi, wr = 2.1e-3, 1.7e-3
    t, pphi, pr = _linear_traj(K, T, wphi, wr, 0.4, 2.9)
    A = 0.7 - 0.3j
    th, ph, scale = 1.1, 0.6, 1.7
    ns = int(T / dt)
    h = oracle.waveform(t, pphi, pr, [mode], np.full((K, 1), A.real), np.full((K, 1), A.imag),
                        th, ph, scale, 0.0, dt, 0, ns)
    ts = np.arange(ns) * dt
    Phi = m * (wphi * ts + 0.4) + n * (wr * ts + 2.9)
    want = A * _m2y2(m, th, ph) * np.exp(-1j * Phi)
    if m > 0:
        want = want + (-1) ** l * np.conj(A) * _m2y2(-m, th, ph) * np.exp(1j * Phi)
    want *= scale
    assert np.max(np.abs(h - want)) < 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("mode", [(3, 1, 2), (3, 3, -1), (5, 2, 0), (4, 0, 3)])
def test_single_mode_closed_form_higher_l(mode):
    """Odd and even l (the (-1)^l of Eq. amp_symmetry) with Y from the pinned harmonics."""
    l, m, n = mode
    T, K, dt = 1.0e5, 7, 23.0
    wphi, wr = 3.3e-3, 2.2e-3
    t, pphi, pr = _linear_traj(K, T, wphi, wr, 1.0, 0.1)
    A = -0.2 + 0.9j
    th, ph = 2.2, 4.4
    ns = int(T / dt)
    h = oracle.waveform(t, pphi, pr, [mode], np.full((K, 1), A.real), np.full((K, 1), A.imag),
                        th, ph, 1.0, 0.0, dt, 0, ns)
    ts = np.arange(ns) * dt
    Phi = m * (wphi * ts + 1.0) + n * (wr * ts + 0.1)
    want = A * oracle.swsh(-2, l, m, th, ph) * np.exp(-1j * Phi)
    if m > 0:
        want = want + (-1) ** l * np.conj(A) * oracle.swsh(-2, l, -m, th, ph) * np.exp(1j * Phi)
    assert np.max(np.abs(h - want)) < 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_shortcut_equals_brute_force_signed_list(seed):
    w = W.tiny_inputs(seed, K=6 + seed, n_samples=300)
    a = oracle.waveform_inputs(w)
    b = oracle.direct_sum(w.t_knots, w.phi_phi, w.phi_r, w.modes, w.amp_re, w.amp_im,
                          w.theta, w.phi, 1.0, w.t0, w.dt, w.n_samples)
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel < 1e-12, rel


def test_brute_force_on_large_phases():
    """Late-inspiral phases (~1e5 rad): reduction in turns agrees with unreduced long double."""
    w = W.config1()
    sub = w.modes[::11]
    idx = np.arange(0, w.N, 11)
    i0 = w.n_samples - 400
    a = oracle.waveform(w.t_knots, w.phi_phi, w.phi_r, sub, w.amp_re[:, idx], w.amp_im[:, idx],
                        w.theta, w.phi, 1.0, 0.0, w.dt, i0, 400)
    b = oracle.direct_sum(w.t_knots, w.phi_phi, w.phi_r, sub, w.amp_re[:, idx], w.amp_im[:, idx],
                          w.theta, w.phi, 1.0, i0 * w.dt, w.dt, 400)
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel < 1e-10, rel


def test_linearity_in_amplitudes_and_scale():
    w1 = W.tiny_inputs(11)
    w2 = W.tiny_inputs(12)
    args = lambda w, ar, ai, s: (w1.t_knots, w1.phi_phi, w1.phi_r, w1.modes, ar, ai, w1.theta,
                                 w1.phi, s, w1.t0, w1.dt, 0, w1.n_samples)
    h1 = oracle.waveform(*args(w1, w1.amp_re, w1.amp_im, 1.0))
    h2 = oracle.waveform(*args(w1, w2.amp_re, w2.amp_im, 1.0))
    h12 = oracle.waveform(*args(w1, w1.amp_re + w2.amp_re, w1.amp_im + w2.amp_im, 1.0))
    assert np.max(np.abs(h12 - h1 - h2)) < 1e-13 * np.max(np.abs(h12))
    h3 = oracle.waveform(*args(w1, w1.amp_re, w1.amp_im, -2.5))
    assert np.max(np.abs(h3 + 2.5 * h1)) < 1e-14 * np.max(np.abs(h3))


def test_sample_window_and_threads_agree():
    w = W.config1()
    full = oracle.waveform_inputs(w, 1000, 3000)
    part = oracle.waveform_inputs(w, 2500, 500, nthreads=4)
    np.testing.assert_array_equal(full[1500:2000], part)


def test_rejects_out_of_range_samples():
    w = W.tiny_inputs(3)
    with pytest.raises(oracle.OracleError):
        oracle.waveform_inputs(w, 0, w.n_samples + 50)


def test_mismatch_definition():
    rng = np.random.default_rng(5)
    a = rng.normal(size=5000) + 1j * rng.normal(size=5000)
    assert oracle.mismatch(a, a) == 0.0
    assert abs(oracle.mismatch(a, 3.0 * a)) < 1e-15
    assert abs(oracle.mismatch(a, -a) - 2.0) < 1e-14
    assert abs(oracle.mismatch(a, 1j * a) - 1.0) < 1e-14
    # a perturbation orthogonal to a: 1 - overlap = 1 - 1/sqrt(1 + e^2)
    d = rng.normal(size=5000) + 1j * rng.normal(size=5000)
    d -= a * (np.vdot(a, d).real / np.vdot(a, a).real)
    d -= 1j * a * (np.vdot(1j * a, d).real / np.vdot(a, a).real)
    e = 1e-3
    b = a + e * d * np.linalg.norm(a) / np.linalg.norm(d)
    want = 1.0 - 1.0 / math.sqrt(1.0 + e * e)
    assert abs(oracle.mismatch(a, b) - want) < 1e-6 * want
    assert abs((1.0 - oracle.overlap(a, b)) - want) < 1e-4 * want


def test_mode_counts_from_paper():
    g = json.load(open(os.path.join(GOLDEN, "mode_counts.json")))
    assert len(W.mode_grid(10, 30)) == g["full_schwarzschild_grid"]["value"]
    ff22 = [(l, m, n) for (l, m, n) in W.mode_grid(10, 30) if l == 2 and m == 2]
    assert len(ff22) == g["ff22_modes"]["value"]
    ns = W.n_samples_for(W.YEAR_S, 10.0)
    assert abs(ns - g["one_year_samples_at_0p1hz"]["approx"]) <= g["one_year_samples_at_0p1hz"]["rel_tol"] * ns
    assert W.n_samples_for(W.WEEK_S, 10.0) == 60480
