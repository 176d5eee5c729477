"""Pins for the oracle's spin-weighted spherical harmonics.

The paper names -2Y_lm as the angular factor of the Schwarzschild sum (Sec. 4) and a utility
module (Sec. 3.D) without giving a formula.  The oracle's Wigner-d sum is pinned by:
textbook closed forms for l = 2, spin 0 reducing to scipy's ordinary harmonics, the addition
theorem, orthonormality by quadrature, the pole values, and the conjugation identity.
"""
import math

import numpy as np
import pytest

import oracle

ANGLES = [(0.3, 1.1), (1.2, 4.0), (2.7, 0.2), (math.pi / 2, 2.5), (0.0, 0.7), (math.pi, 5.9)]


def _m2y2(m, th, ph):
    c, s = math.cos(th), math.sin(th)
    amp = {2: math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2,
           1: math.sqrt(5 / (16 * math.pi)) * s * (1 + c),
           0: math.sqrt(15 / (32 * math.pi)) * s * s,
           -1: math.sqrt(5 / (16 * math.pi)) * s * (1 - c),
           -2: math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2}[m]
    return amp * complex(math.cos(m * ph), math.sin(m * ph))


@pytest.mark.parametrize("th,ph", ANGLES)
@pytest.mark.parametrize("m", [-2, -1, 0, 1, 2])
def test_l2_closed_forms(m, th, ph):
    assert abs(oracle.swsh(-2, 2, m, th, ph) - _m2y2(m, th, ph)) < 1e-15


def test_spin0_is_scipy_sph_harm():
    sp = pytest.importorskip("scipy.special")
    f = getattr(sp, "sph_harm_y", None)
    for l in range(0, 11):
        for m in range(-l, l + 1):
            for th, ph in ANGLES[:4]:
                if f is not None:
                    ref = complex(f(l, m, th, ph))
                else:  # older scipy: sph_harm(m, l, azimuth, polar)
                    ref = complex(sp.sph_harm(m, l, ph, th))
                got = oracle.swsh(0, l, m, th, ph)
                assert abs(got - ref) < 1e-13 * max(1.0, abs(ref)), (l, m, th)


@pytest.mark.parametrize("l", range(2, 11))
def test_addition_theorem(l):
    for th, ph in ANGLES:
        tot = sum(abs(oracle.swsh(-2, l, m, th, ph)) ** 2 for m in range(-l, l + 1))
        assert abs(tot - (2 * l + 1) / (4 * math.pi)) < 1e-13


def test_orthonormality_by_quadrature():
    x, wx = np.polynomial.legendre.leggauss(40)
    th = np.arccos(x)
    nph = 32
    ph = 2 * math.pi * np.arange(nph) / nph
    wph = 2 * math.pi / nph
    lm = [(l, m) for l in range(2, 7) for m in range(-l, l + 1)]
    Y = np.array([[[oracle.swsh(-2, l, m, a, b) for b in ph] for a in th] for (l, m) in lm])
    G = np.einsum("iab,jab,a->ij", np.conj(Y), Y, wx) * wph
    np.testing.assert_allclose(G, np.eye(len(lm)), atol=1e-12)


@pytest.mark.parametrize("l", range(2, 11))
def test_pole_values(l):
    """At theta = 0 only m = 2 survives for spin -2; at theta = pi only m = -2."""
    ph = 0.9
    for m in range(-l, l + 1):
        y0 = oracle.swsh(-2, l, m, 0.0, ph)
        yp = oracle.swsh(-2, l, m, math.pi, ph)
        if m == 2:
            want = math.sqrt((2 * l + 1) / (4 * math.pi)) * complex(math.cos(2 * ph), math.sin(2 * ph))
            assert abs(y0 - want) < 1e-14
        else:
            assert abs(y0) < 1e-14
        if m != -2:
            assert abs(yp) < 1e-14
        else:
            assert abs(abs(yp) - math.sqrt((2 * l + 1) / (4 * math.pi))) < 1e-14


@pytest.mark.parametrize("l", [2, 3, 5, 10])
def test_conjugation_identity(l):
    """conj(sY_lm) = (-1)^(s+m) (-s)Y_l,-m."""
    for th, ph in ANGLES[:4]:
        for m in range(-l, l + 1):
            lhs = np.conj(oracle.swsh(-2, l, m, th, ph))
            rhs = (-1) ** (-2 + m) * oracle.swsh(2, l, -m, th, ph)
            assert abs(lhs - rhs) < 1e-14
