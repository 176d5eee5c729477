"""Pins for the oracle's Mode Selector (Sec. 3.D).

* exact definition: powers, ordering, cumulative sums and the (1 - eps) cut recomputed with
  rational arithmetic (fractions) on random inputs;
* a closed form: geometric powers r^j give a kept count of ceil(log(eps + (1-eps) r^N)/log r);
* the union over knots, the eps -> 0 and eps >= 1 limits, and the m > 0 doubling.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _exact(amp_re, amp_im, m, eps):
    K, N = amp_re.shape
    keep = np.zeros(N, dtype=bool)
    e = Fraction(eps)
    for k in range(K):
        p = []
        for i in range(N):
            v = Fraction(float(amp_re[k, i])) ** 2 + Fraction(float(amp_im[k, i])) ** 2
            p.append((v * (2 if m[i] > 0 else 1), i))
        p.sort(key=lambda x: (-x[0], x[1]))
        total = sum(v for v, _ in p)
        if total == 0:
            continue
        c = Fraction(0)
        for v, i in p:
            c += v
            keep[i] = True
            if c >= (1 - e) * total:
                break
    return keep


@pytest.mark.parametrize("seed", range(6))
def test_matches_exact_rational_definition(seed):
    rng = np.random.default_rng(seed)
    K, N = 5, 40
    scale = 10.0 ** rng.uniform(-4, 0, size=N)
    re = rng.normal(size=(K, N)) * scale
    im = rng.normal(size=(K, N)) * scale
    modes = np.stack([np.full(N, 2), rng.integers(0, 3, size=N), np.arange(N)], axis=1)
    for eps in (1e-1, 1e-3, 1e-6):
        got = oracle.mode_select(re, im, modes, eps)
        want = _exact(re, im, modes[:, 1], eps)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("r,N,eps", [(0.5, 40, 1e-3), (0.8, 60, 1e-5), (0.9, 200, 1e-2)])
def test_geometric_closed_form(r, N, eps):
    p = r ** np.arange(N)
    re = np.sqrt(p)[None, :]
    im = np.zeros_like(re)
    modes = np.stack([np.full(N, 2), np.zeros(N, int), np.arange(N)], axis=1)
    kept = oracle.mode_select(re, im, modes, eps)
    want = math.ceil(math.log(eps + (1 - eps) * r ** N) / math.log(r))
    assert kept.sum() == want
    assert np.all(kept[:want]) and not np.any(kept[want:])


def test_union_and_limits_and_doubling():
    N = 6
    modes = np.stack([np.full(N, 2), np.array([0, 0, 0, 1, 0, 0]), np.arange(N)], axis=1)
    re = np.array([[3.0, 0.1, 0.0, 0.0, 0.0, 0.2],
                   [0.0, 0.0, 5.0, 0.1, 0.0, 0.0]])
    im = np.zeros_like(re)
    # eps large: only the top mode of each knot, and their union
    np.testing.assert_array_equal(oracle.mode_select(re, im, modes, 2.0),
                                  [True, False, True, False, False, False])
    # eps -> 0: every mode with nonzero power at some knot
    np.testing.assert_array_equal(oracle.mode_select(re, im, modes, 0.0),
                                  [True, True, True, True, False, True])
    # m > 0 counts twice: mode 3 (m = 1) outranks mode 1 at equal amplitude
    re2 = np.array([[1.0, 0.5, 0.0, 0.5, 0.0, 0.0]])
    got = oracle.mode_select(re2, np.zeros_like(re2), modes, 0.3)
    np.testing.assert_array_equal(got, [True, False, False, True, False, False])
