"""Pins for the oracle's not-a-knot cubic spline (Sec. 3.C).

Each check is independent of the oracle's own formula: exact reproduction of cubics (the
not-a-knot spline is exact on any cubic), the unique Lagrange cubic for K = 4, the spline's
defining conditions (interpolation, C2, continuous third derivative at t_1 and t_{K-2}),
fourth-order convergence, and scipy's CubicSpline(bc_type='not-a-knot') as a library
cross-check.
"""
import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import workloads as W


def _rand_knots(rng, K, T=1.0e6):
    gaps = rng.uniform(0.2, 1.0, size=K - 1)
    t = np.concatenate([[0.0], np.cumsum(gaps)])
    return t / t[-1] * T


def _poly_at(c, t):
    return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]


@pytest.mark.parametrize("K", [4, 5, 7, 12, 40, 100])
def test_reproduces_cubics_exactly(K):
    rng = np.random.default_rng(K)
    t = _rand_knots(rng, K, T=10.0)
    c = rng.normal(size=4)
    y = _poly_at(c, t)
    coef = oracle.spline_nak(t, y)
    x = np.sort(rng.uniform(t[0], t[-1], size=500))
    got = oracle.spline_eval(t, coef, x)
    want = _poly_at(c, x)
    scale = np.max(np.abs(y))
    assert np.max(np.abs(got - want)) <= 1e-12 * scale


def test_reproduces_quadratic_amplitudes_on_config_grid():
    """The synthetic amplitudes are quadratic in t: the spline must equal the closed form."""
    w = W.config1()
    x = np.linspace(0.0, w.T, 3001)
    Aexact = w.amp_model(x)
    for i in [0, 17, 60, 131]:
        for arr, want in ((w.amp_re, Aexact.real), (w.amp_im, Aexact.imag)):
            coef = oracle.spline_nak(w.t_knots, arr[:, i])
            got = oracle.spline_eval(w.t_knots, coef, x)
            assert np.max(np.abs(got - want[:, i])) <= 1e-12 * np.max(np.abs(arr[:, i]))


def test_k4_is_the_lagrange_cubic():
    rng = np.random.default_rng(4)
    t = np.array([0.0, 0.3, 1.1, 2.0])
    y = rng.normal(size=4)
    coef = oracle.spline_nak(t, y)
    x = np.linspace(0.0, 2.0, 101)
    lag = np.zeros_like(x)
    for j in range(4):
        b = np.ones_like(x)
        for k in range(4):
            if k != j:
                b *= (x - t[k]) / (t[j] - t[k])
        lag += y[j] * b
    got = oracle.spline_eval(t, coef, x)
    np.testing.assert_allclose(got, lag, rtol=0, atol=1e-13)


def _derivs(coef, h):
    """Value, 1st, 2nd, 3rd derivative at both ends of each segment (local x)."""
    c0, c1, c2, c3 = coef.T
    left = np.stack([c0, c1, 2 * c2, 6 * c3])
    right = np.stack([c0 + c1 * h + c2 * h ** 2 + c3 * h ** 3,
                      c1 + 2 * c2 * h + 3 * c3 * h ** 2,
                      2 * c2 + 6 * c3 * h, 6 * c3])
    return left, right


@pytest.mark.parametrize("K", [5, 9, 30])
def test_defining_conditions(K):
    rng = np.random.default_rng(100 + K)
    t = _rand_knots(rng, K, T=3.0)
    y = rng.normal(size=K)
    coef = oracle.spline_nak(t, y)
    h = np.diff(t)
    left, right = _derivs(coef, h)
    # interpolation at every knot
    np.testing.assert_allclose(left[0], y[:-1], atol=1e-14)
    np.testing.assert_allclose(right[0], y[1:], atol=1e-12)
    # C1 and C2 at interior knots
    np.testing.assert_allclose(right[1][:-1], left[1][1:], atol=1e-10)
    np.testing.assert_allclose(right[2][:-1], left[2][1:], atol=1e-9)
    # not-a-knot: third derivative continuous at t_1 and t_{K-2}
    s3 = 6 * coef[:, 3]
    tol = 1e-8 * np.max(np.abs(s3))
    assert abs(s3[0] - s3[1]) <= tol
    assert abs(s3[-1] - s3[-2]) <= tol


def test_fourth_order_convergence():
    errs = []
    for K in (20, 40, 80, 160):
        t = np.linspace(0.0, 3.0, K) + 0.1 * np.sin(np.linspace(0.0, 7.0, K)) * (3.0 / K)
        y = np.sin(2.0 * t) * np.exp(0.3 * t)
        coef = oracle.spline_nak(t, y)
        x = np.linspace(0.0, 3.0, 4001)
        errs.append(np.max(np.abs(oracle.spline_eval(t, coef, x) - np.sin(2 * x) * np.exp(0.3 * x))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.6), rates


@pytest.mark.parametrize("K", [4, 6, 25, 100, 300])
def test_matches_scipy_not_a_knot(K):
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(7 + K)
    t = W.knot_times(1.0e7, K)
    y = rng.normal(size=K) * 10.0 ** rng.uniform(-3, 3)
    coef = oracle.spline_nak(t, y)
    cs = interp.CubicSpline(t, y, bc_type="not-a-knot")
    # scipy stores c[3-p, k] for the power p in local x
    ref = cs.c[::-1].T
    for p in range(4):
        scale = np.max(np.abs(ref[:, p])) + 1e-300
        assert np.max(np.abs(coef[:, p] - ref[:, p])) <= 1e-10 * scale, p


def test_rejects_degenerate_knots():
    with pytest.raises(oracle.OracleError):
        oracle.spline_nak([0.0, 1.0, 2.0], [1.0, 2.0, 3.0])
    with pytest.raises(oracle.OracleError):
        oracle.spline_nak([0.0, 1.0, 1.0, 2.0, 3.0], [1.0, 2.0, 3.0, 4.0, 5.0])
