"""The summation's division of work among CTAs (host planning, no GPU).

few_plan_cta_slices is the function few_waveform and few_batch_plan use.  Checked here against
an independent description of its contract: contiguous slices in (waveform, sample) order that
cover every sample once, starting only at pass boundaries (a pass = `pass` consecutive samples
of one segment), with costs (passes x (slots + 16)) balanced to within one pass.
"""
import math

import numpy as np
import pytest

from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import workloads as W


def _passes(seg, a, b, P):
    """Passes a slice [a, b) of one waveform runs: per segment, ceil(overlap / P)."""
    n = 0
    for s in range(len(seg) - 1):
        lo, hi = max(a, seg[s]), min(b, seg[s + 1])
        if hi > lo:
            n += math.ceil((hi - lo) / P)
    return n


def _is_pass_boundary(seg, x, P):
    if x == seg[-1]:
        return True
    s = int(np.searchsorted(seg, x, side="right")) - 1
    return (x - seg[s]) % P == 0


def _slice_costs(segs, slots, wv, sm, P):
    """Cost of every slice, walking (wave, sample) order."""
    costs = []
    for g in range(len(wv) - 1):
        w0, s0, w1, s1 = int(wv[g]), int(sm[g]), int(wv[g + 1]), int(sm[g + 1])
        c, w, a = 0, w0, s0
        while (w, a) < (w1, s1) and w < len(segs):
            end = s1 if w == w1 else int(segs[w][-1])
            c += _passes(segs[w], a, end, P) * (slots[w] + 16)
            w, a = w + 1, 0
        costs.append(c)
    return np.array(costs)


def _check(segs, slots, grid, P):
    wv, sm = F.few_plan_cta_slices(segs, slots, grid, P)
    assert (wv[0], sm[0]) == (0, 0) and (wv[-1], sm[-1]) == (len(segs), 0)
    pairs = list(zip(wv.tolist(), sm.tolist()))
    assert pairs == sorted(pairs), "slices out of order"
    for w, x in pairs[:-1]:
        assert 0 <= w < len(segs) and 0 <= x <= segs[w][-1]
        assert _is_pass_boundary(segs[w], x, P), (w, x)
    costs = _slice_costs(segs, slots, wv, sm, P)
    total = sum(_passes(s, 0, int(s[-1]), P) * (c + 16) for s, c in zip(segs, slots))
    assert costs.sum() == total  # every pass in exactly one slice
    one = max(c + 16 for c in slots)  # the largest cost of one pass
    ideal = total / grid
    assert costs.max() <= ideal + one and costs.min() >= ideal - one, (costs.min(), costs.max(), ideal)
    return costs


@pytest.mark.parametrize("grid,P", [(304, 1024), (152, 2048)])
def test_one_year_waveform_slices(grid, P):
    """The one-year waveform at R = 4 x 256 threads on 2 CTAs per SM and at the default R = 8 x
    256 threads on one CTA per SM: 10 or 11 passes per CTA (equal-sample slices reached 13)."""
    w = W.config2()
    seg = F.few_plan_segments(w.t_knots, w.t0, w.dt, w.n_samples)
    costs = _check([seg], [1281], grid, P)
    assert sorted(set((costs // 1297).tolist())) == [10, 11]


@pytest.mark.parametrize("grid,P", [(304, 1024), (304, 2048), (152, 512), (152, 2048), (608, 1024)])
def test_batch_of_uneven_waveforms(grid, P):
    rng = np.random.default_rng(11 + grid + P)
    segs, slots = [], []
    for k in range(12):
        K = int(rng.integers(4, 160))
        T = float(rng.uniform(1e5, 3e7))
        dt = float(rng.choice([2.0, 5.0, 10.0, 15.0]))
        t = T * (1.0 - (1.0 - np.arange(K) / (K - 1)) ** 2)
        n = int(min(T // dt, 4_000_000))
        segs.append(F.few_plan_segments(t, 0.0, dt, n))
        slots.append(int(rng.integers(1, 2000)))
    _check(segs, slots, grid, P)


def test_more_ctas_than_passes():
    t = np.linspace(0.0, 100.0, 5)
    seg = F.few_plan_segments(t, 0.0, 1.0, 50)
    wv, sm = F.few_plan_cta_slices([seg], [7], 64, 1024)
    assert (wv[-1], sm[-1]) == (1, 0)
    # a handful of passes among 64 CTAs: most slices empty, every start still a pass boundary
    for w, x in zip(wv[:-1], sm[:-1]):
        assert w == 1 or _is_pass_boundary(seg, int(x), 1024)


def test_rejects_bad_arguments():
    seg = np.array([0, 10, 20], dtype=np.int64)
    for args in (([seg], [5], 0, 128), ([seg], [5], 4, 0), ([seg], [0], 4, 128),
                 ([np.array([0, 10, 5], dtype=np.int64)], [5], 4, 128)):
        with pytest.raises(F.FewError):
            F.few_plan_cta_slices(*args)
