"""Mode Selector (Sec. 3.D) on the GPU against the oracle.

The selection is integer output decided by FP64 cumulative sums; the GPU sums in a parallel
order, so the masks must be equal except for modes whose cumulative power at some knot lies within
rounding (1e-12 relative) of the cut -- each such disagreement is checked to be one (for eps > 0
there are at most a couple; eps = 0 turns every mode below one ulp of the total into one).
"""
import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu_select(ctx, amp_re, amp_im, modes, eps):
    import torch
    re = torch.as_tensor(np.ascontiguousarray(amp_re)).cuda()
    im = torch.as_tensor(np.ascontiguousarray(amp_im)).cuda()
    mask = torch.empty(re.shape[1], dtype=torch.uint8, device="cuda")
    F.few_mode_select(ctx.handle, re, im, np.asarray(modes)[:, 1], eps, mask, RT.current_stream())
    torch.cuda.synchronize()
    return mask.cpu().numpy().astype(bool)


def _near_cut(amp_re, amp_im, modes, eps, i):
    """True if mode i sits within rounding of the cut at some knot (either decision is valid)."""
    m = np.asarray(modes)[:, 1]
    for k in range(amp_re.shape[0]):
        p = amp_re[k] ** 2 + amp_im[k] ** 2
        p = np.where(m > 0, 2 * p, p)
        order = np.lexsort((np.arange(len(p)), -p))
        c = np.cumsum(p[order])
        tgt = (1 - eps) * c[-1]
        r = int(np.where(order == i)[0][0])
        before = c[r - 1] if r > 0 else 0.0
        if abs(before - tgt) <= 1e-12 * c[-1]:
            return True
    return False


@pytest.mark.parametrize("cfg,eps", [("week", 1e-5), ("year", 1e-5), ("year", 1e-2),
                                     ("year", 1e-9), ("year", 0.0)])
def test_mode_select_matches_oracle(gpu_ctx, cfg, eps):
    w = W.config1() if cfg == "week" else W.config2()
    g = _gpu_select(gpu_ctx, w.amp_re, w.amp_im, w.modes, eps)
    o = oracle.mode_select(w.amp_re, w.amp_im, w.modes, eps)
    diff = np.where(g != o)[0]
    for i in diff:
        assert _near_cut(w.amp_re, w.amp_im, w.modes, eps, i), i
    if eps > 0.0:
        assert len(diff) <= 2
    # eps = 0 makes every mode whose power is below one ulp of the running sum a rounding
    # decision, so only the per-mode check above applies there


def test_mode_select_edge_cases(gpu_ctx):
    # zero-power knot keeps nothing; one mode; exact ties ordered by mode index
    modes = np.array([[2, 0, 0], [2, 0, 1], [2, 0, 2]])
    re = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]])
    im = np.zeros_like(re)
    np.testing.assert_array_equal(_gpu_select(gpu_ctx, re, im, modes, 0.5), [True, True, False])
    np.testing.assert_array_equal(_gpu_select(gpu_ctx, re[:1], im[:1], modes, 0.5), [False] * 3)
    one = np.array([[2, 2, 0]])
    np.testing.assert_array_equal(_gpu_select(gpu_ctx, np.ones((3, 1)), np.zeros((3, 1)), one, 0.1),
                                  [True])
    with pytest.raises(F.FewError):
        _gpu_select(gpu_ctx, re, im, modes, -1.0)


@pytest.mark.parametrize("N", [1, 2, 31, 127, 128, 129, 255, 257, 1000, 2049, 4096])
def test_mode_select_ragged_exact(gpu_ctx, N):
    # integer powers with many exact ties: every prefix sum is exact in FP64, so the cut and the
    # tie order (lower mode index first) are unique and the masks must agree bit for bit
    rng = np.random.default_rng(1000 + N)
    modes = np.stack([np.full(N, 2), rng.integers(0, 3, N), np.zeros(N, int)], axis=1)
    re = rng.integers(0, 4, (5, N)).astype(np.float64)
    im = rng.integers(0, 3, (5, N)).astype(np.float64)
    for eps in (0.5, 0.1, 1e-3, 0.0):
        g = _gpu_select(gpu_ctx, re, im, modes, eps)
        o = oracle.mode_select(re, im, modes, eps)
        np.testing.assert_array_equal(g, o, err_msg=f"N={N} eps={eps}")


@pytest.mark.parametrize("N", [129, 2049, 4096])
def test_mode_select_ragged_random(gpu_ctx, N):
    rng = np.random.default_rng(2000 + N)
    modes = np.stack([np.full(N, 2), rng.integers(0, 3, N), np.zeros(N, int)], axis=1)
    re = rng.standard_normal((7, N)) * np.exp(-3.0 * rng.random(N))
    im = rng.standard_normal((7, N)) * np.exp(-3.0 * rng.random(N))
    eps = 1e-4
    g = _gpu_select(gpu_ctx, re, im, modes, eps)
    o = oracle.mode_select(re, im, modes, eps)
    diff = np.where(g != o)[0]
    assert len(diff) <= 2
    for i in diff:
        assert _near_cut(re, im, modes, eps, i), i
