"""Pins for the oracle's direct (non-interpolated) summation (Sec. 3.C).

* with the arrays taken from the spline-free closed forms of a single mode (constant amplitude,
  linear phases), the direct sum equals the analytic h (l = 2 textbook harmonics);
* fed with the interpolating splines' own values at the samples, it equals the interpolated
  summation (two routes to the same sum);
* linear in the amplitudes.
"""
import math

import numpy as np

import oracle
from paper_2104_04582_gb300 import workloads as W


def _m2y2(m, th, ph):
    c, s = math.cos(th), math.sin(th)
    amp = {2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
           1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c),
           0: math.sqrt(15 / (32 * math.pi)) * s * s,
           -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
           -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2}[m]
    return amp * complex(math.cos(m * ph), math.sin(m * ph))


def test_single_mode_closed_form():
    ts = np.arange(4000) * 17.0
    pphi, pr = 2.1e-3 * ts + 0.4, 1.7e-3 * ts + 2.9
    A = 0.3 + 0.8j
    for (l, m, n) in ((2, 2, 3), (2, 1, -2), (2, 0, 1)):
        h = oracle.direct_dense(pphi, pr, [(l, m, n)], np.full((len(ts), 1), A.real),
                                np.full((len(ts), 1), A.imag), 0.9, 2.2, 1.5)
        Phi = m * pphi + n * pr
        want = A * _m2y2(m, 0.9, 2.2) * np.exp(-1j * Phi)
        if m > 0:
            want = want + (-1) ** l * np.conj(A) * _m2y2(-m, 0.9, 2.2) * np.exp(1j * Phi)
        assert np.max(np.abs(h - 1.5 * want)) < 1e-12 * np.max(np.abs(want))


def test_equals_interpolated_sum_on_spline_values():
    w = W.tiny_inputs(9, K=10, n_samples=700)
    ts = w.t0 + np.arange(w.n_samples) * w.dt
    pphi = oracle.spline_eval(w.t_knots, oracle.spline_nak(w.t_knots, w.phi_phi), ts)
    pr = oracle.spline_eval(w.t_knots, oracle.spline_nak(w.t_knots, w.phi_r), ts)
    ar = np.stack([oracle.spline_eval(w.t_knots, oracle.spline_nak(w.t_knots, w.amp_re[:, i]), ts)
                   for i in range(w.N)], axis=1)
    ai = np.stack([oracle.spline_eval(w.t_knots, oracle.spline_nak(w.t_knots, w.amp_im[:, i]), ts)
                   for i in range(w.N)], axis=1)
    d = oracle.direct_dense(pphi, pr, w.modes, ar, ai, w.theta, w.phi)
    h = oracle.waveform_inputs(w)
    assert np.linalg.norm(d - h) <= 1e-11 * np.linalg.norm(h)


def test_linear_in_amplitudes():
    rng = np.random.default_rng(2)
    ns, N = 300, 5
    modes = np.array([(2, 2, 0), (3, 1, 1), (2, 0, -1), (4, 3, 2), (5, 5, -3)])
    pphi, pr = rng.uniform(0, 1e4, ns), rng.uniform(0, 1e4, ns)
    a1, b1, a2, b2 = (rng.normal(size=(ns, N)) for _ in range(4))
    h1 = oracle.direct_dense(pphi, pr, modes, a1, b1, 0.4, 1.0)
    h2 = oracle.direct_dense(pphi, pr, modes, a2, b2, 0.4, 1.0)
    h12 = oracle.direct_dense(pphi, pr, modes, a1 + a2, b1 + b2, 0.4, 1.0)
    assert np.max(np.abs(h12 - h1 - h2)) < 1e-13 * np.max(np.abs(h12))
