"""Pin for the oracle's per-sample orbital phases (reduced modulo 2 pi, in turns).

A phase that is exactly a cubic in t is reproduced by the not-a-knot spline; with dyadic knot
times and coefficients the knot values are exact doubles, so the reduced phase has an exact
value computable with rational arithmetic and a 40-digit 2 pi.  Magnitudes reach 1e5-1e7 rad,
as the one- and four-year phases do.
"""
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle

getcontext().prec = 50
TWO_PI = Fraction(Decimal("6.2831853071795864769252867665590057683943387987502"))


def _exact_turns(c, t):
    x = Fraction(t)
    v = ((Fraction(c[3]) * x + Fraction(c[2])) * x + Fraction(c[1])) * x + Fraction(c[0])
    turns = v / TWO_PI
    return float(turns - round(turns))


@pytest.mark.parametrize("scale", [1e3, 1e5, 1.6e7])
def test_reduced_phases_of_an_exact_cubic(scale):
    T = 2.0 ** 20
    t = np.array([0.0, 2.0 ** 14, 2.0 ** 16, 2.0 ** 17, 2.0 ** 18, 2.0 ** 19, 2.0 ** 20])
    # coefficients chosen so that every knot value is an exact double
    c = [0.75, scale / T, 2.0 ** -30, 2.0 ** -52]
    y = np.array([float(((Fraction(c[3]) * Fraction(v) + Fraction(c[2])) * Fraction(v)
                         + Fraction(c[1])) * Fraction(v) + Fraction(c[0])) for v in t])
    for v, yy in zip(t, y):
        exact = ((Fraction(c[3]) * Fraction(v) + Fraction(c[2])) * Fraction(v)
                 + Fraction(c[1])) * Fraction(v) + Fraction(c[0])
        assert Fraction(yy) == exact
    dt = 1024.0  # exact sample times i*dt, the last one on the last knot
    ts = np.arange(1025) * dt
    got = oracle.phases(t, y, -y, 0.0, dt, 0, len(ts))
    want = np.array([_exact_turns(c, float(v)) for v in ts])
    d = got[:, 0] - want
    d -= np.round(d)
    assert np.max(np.abs(d)) < 1e-12
    d2 = got[:, 1] + want
    d2 -= np.round(d2)
    assert np.max(np.abs(d2)) < 1e-12
