"""Mode Selector (Sec. 3.D) on the GPU against the oracle.

The selection is integer output decided by FP64 cumulative sums.  Both sides form each power as
fl(fl(re^2) + fl(im^2)) and each cumulative sum left to right over the sorted powers, so the
masks must agree bit for bit: for every workload, every eps (including eps = 0, where the cut is
where the running sum stops changing), and ragged mode counts.
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


@pytest.mark.parametrize("cfg,eps", [("week", 1e-5), ("year", 1e-5), ("year", 1e-2),
                                     ("year", 1e-9), ("year", 0.0)])
def test_mode_select_matches_oracle(gpu_ctx, cfg, eps):
    w = W.config1() if cfg == "week" else W.config2()
    g = _gpu_select(gpu_ctx, w.amp_re, w.amp_im, w.modes, eps)
    o = oracle.mode_select(w.amp_re, w.amp_im, w.modes, eps)
    np.testing.assert_array_equal(g, o, err_msg=f"{cfg} eps={eps}")


@pytest.mark.parametrize("seed", range(4))
def test_mode_select_batch_workload_exact(gpu_ctx, seed):
    # the batch workload's per-waveform decay scales spread the powers over many decades, so the
    # running sum stops changing at different ranks of different knots
    rng = np.random.default_rng(3000 + seed)
    sigma_l = float(np.exp(rng.uniform(np.log(0.5), np.log(8.0))))
    sigma_n = float(np.exp(rng.uniform(np.log(1.0), np.log(60.0))))
    w = W.make_inputs(0.25 * W.YEAR_S, int(rng.integers(50, 151)), 10.0, W.mode_grid(10, 30),
                      3000 + seed, sigma_l, sigma_n)
    for eps in (1e-2, 1e-5, 1e-9, 1e-14, 0.0):
        g = _gpu_select(gpu_ctx, w.amp_re, w.amp_im, w.modes, eps)
        o = oracle.mode_select(w.amp_re, w.amp_im, w.modes, eps)
        np.testing.assert_array_equal(g, o, err_msg=f"seed={seed} eps={eps}")


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


@pytest.mark.parametrize("N", [129, 2049, 3843, 4096])
def test_mode_select_ragged_random(gpu_ctx, N):
    rng = np.random.default_rng(2000 + N)
    modes = np.stack([np.full(N, 2), rng.integers(0, 3, N), np.zeros(N, int)], axis=1)
    re = rng.standard_normal((7, N)) * np.exp(-3.0 * rng.random(N))
    im = rng.standard_normal((7, N)) * np.exp(-3.0 * rng.random(N))
    for eps in (1e-4, 1e-12, 0.0, 1.0, 2.0):
        g = _gpu_select(gpu_ctx, re, im, modes, eps)
        o = oracle.mode_select(re, im, modes, eps)
        np.testing.assert_array_equal(g, o, err_msg=f"N={N} eps={eps}")


def test_mode_select_decades_exact(gpu_ctx):
    # powers spread over 300 decades (the running sum stops changing early) and equal powers
    # that only the mode index orders
    N = 3000
    rng = np.random.default_rng(77)
    modes = np.stack([np.full(N, 2), rng.integers(0, 3, N), np.zeros(N, int)], axis=1)
    re = 10.0 ** rng.uniform(-150, 0, (4, N))
    im = np.zeros((4, N))
    re[:, ::7] = 0.25
    for eps in (1e-3, 1e-15, 0.0):
        g = _gpu_select(gpu_ctx, re, im, modes, eps)
        o = oracle.mode_select(re, im, modes, eps)
        np.testing.assert_array_equal(g, o, err_msg=f"eps={eps}")


def _tie_knots(N, rng):
    # Powers a^2 + b^2 in units of 2^-54 beside a leading power 1: 2 (exactly half an ulp of the
    # running sum 1, a rounding tie decided by the parity of the sum), 5 (above half), 1 (below
    # half) and 8 (a whole ulp).  Every power and every product is exact, so the masks depend only
    # on how each addition rounds.
    ab = np.array([[1, 1], [1, 2], [0, 1], [2, 2]])
    pick = rng.integers(0, 4, (3, N))
    re, im = ab[pick, 0] * 2.0 ** -27, ab[pick, 1] * 2.0 ** -27
    re[:, 0], im[:, 0] = 1.0, 0.0
    return re, im


@pytest.mark.parametrize("N", [40, 300, 3843])
def test_mode_select_rounding_ties_exact(gpu_ctx, N):
    # few ties (N = 40) stay inside the block-wide scan; hundreds of ties also run the sequential
    # chain that finishes the sums after the scan's round limit
    rng = np.random.default_rng(4000 + N)
    re, im = _tie_knots(N, rng)
    modes = np.stack([np.full(N, 2), np.zeros(N, int), np.zeros(N, int)], axis=1)
    for eps in (1e-16, 1e-17, 0.0):
        g = _gpu_select(gpu_ctx, re, im, modes, eps)
        o = oracle.mode_select(re, im, modes, eps)
        np.testing.assert_array_equal(g, o, err_msg=f"N={N} eps={eps}")


def test_mode_select_subnormal_and_infinite_powers(gpu_ctx):
    # subnormal powers (sums of multiples of 2^-1074, then crossing into the normal range), and a
    # knot with an infinite power, which the cut reaches at its first rank
    N = 1500
    rng = np.random.default_rng(4100)
    modes = np.stack([np.full(N, 2), rng.integers(0, 3, N), np.zeros(N, int)], axis=1)
    re = 10.0 ** rng.uniform(-162, -154, (4, N))
    im = 10.0 ** rng.uniform(-163, -160, (4, N))
    re[1, :3] = [1e-150, 3e-151, 2e-152]
    re[3, 17] = 1e200
    for eps in (1e-3, 1e-12, 0.0):
        g = _gpu_select(gpu_ctx, re, im, modes, eps)
        o = oracle.mode_select(re, im, modes, eps)
        np.testing.assert_array_equal(g, o, err_msg=f"eps={eps}")
