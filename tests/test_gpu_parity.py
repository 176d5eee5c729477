"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Sizes: the one-week workload in full (60,480 samples x 132 modes, many passes and segments, a
ragged tail), the one-year 3843-mode workload at full size in the benchmark's launch
configuration (oracle on windows at the start, across knots, and at the end), the four-year
workload's mixed path on a 1e5-sample window, and tiny cases with ragged sample counts.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W
from tests.gpu_common import (FP64_PHASE, FP64_REL_L2, MIXED_MISMATCH, max_phase_err,
                              oracle_threads, rel_l2, to_host)

pytestmark = pytest.mark.gpu


def _gpu(ctx, w, prec, c64=None, device_data=True, **kw):
    import torch
    tr = RT.from_inputs(ctx, w, device_data=device_data)
    out = RT.waveform_inputs(ctx, tr, w, prec, c64, **kw)
    torch.cuda.synchronize()
    assert ctx.sync_status() == F.FEW_OK
    h = to_host(out)
    tr.release()
    return h


def _oracle(w, i_begin=0, count=None):
    return oracle.waveform_inputs(w, i_begin, count, nthreads=oracle_threads())


def test_week_fp64_full(gpu_ctx):
    w = W.config1()
    g = _gpu(gpu_ctx, w, F.FEW_FP64)
    o = _oracle(w)
    assert rel_l2(g, o) <= FP64_REL_L2
    assert max_phase_err(g, o) <= FP64_PHASE


def test_week_mixed_full(gpu_ctx):
    w = W.config1()
    g = _gpu(gpu_ctx, w, F.FEW_MIXED)
    o = _oracle(w)
    mm = oracle.mismatch(g, o)
    assert mm <= MIXED_MISMATCH, mm
    # stated expectation for FP32 amplitudes and exponentials: well below the gate
    assert rel_l2(g, o) <= 1e-4
    assert max_phase_err(g, o) <= 1e-3


@pytest.fixture(scope="module")
def year():
    return W.config2()


def _windows(w):
    ns = w.n_samples
    seg = F.few_plan_segments(w.t_knots, w.t0, w.dt, ns)
    mid = int(seg[len(seg) // 2]) - 1000          # straddles a knot
    late = int(seg[-3]) - 700                      # short late segments
    return [(0, 2000), (mid, 2000), (late, 1500), (ns - 1700, 1700)]


def test_year_fp64_windows(gpu_ctx, year):
    g = _gpu(gpu_ctx, year, F.FEW_FP64)
    assert g.shape[0] == year.n_samples
    for i0, n in _windows(year):
        o = _oracle(year, i0, n)
        assert rel_l2(g[i0:i0 + n], o) <= FP64_REL_L2, (i0, rel_l2(g[i0:i0 + n], o))
        assert max_phase_err(g[i0:i0 + n], o) <= FP64_PHASE, i0


def test_year_mixed_windows_and_full_series(gpu_ctx, year):
    gm = _gpu(gpu_ctx, year, F.FEW_MIXED)
    for i0, n in _windows(year):
        o = _oracle(year, i0, n)
        assert oracle.mismatch(gm[i0:i0 + n], o) <= MIXED_MISMATCH, i0
    g64 = _gpu(gpu_ctx, year, F.FEW_FP64)
    assert oracle.mismatch(gm, g64) <= MIXED_MISMATCH


def _mismatch_on_device(a, b) -> float:
    """1 - overlap (unit noise, no maximisation) of two device series, in FP64 on the GPU."""
    import torch
    a = a.to(torch.complex128)
    b = b.to(torch.complex128)
    ab = torch.sum(torch.conj(a) * b).real
    aa = torch.sum(torch.abs(a) ** 2)
    bb = torch.sum(torch.abs(b) ** 2)
    return float(1.0 - ab / torch.sqrt(aa * bb))


def test_four_year_mixed_window_and_full_series(gpu_ctx):
    """The stress workload (4 yr at dt = 2 s, 63,115,200 samples, K = 300, 3843 modes): the mixed
    path against the oracle on a 1e5-sample window at the end and on the first 2000 samples, and
    by mismatch over the full series against the FP64 GPU path (itself checked against the
    oracle on the same windows)."""
    import torch
    w = W.config5()
    tr = RT.from_inputs(gpu_ctx, w)
    gm = RT.waveform_inputs(gpu_ctx, tr, w, F.FEW_MIXED)
    g64 = RT.waveform_inputs(gpu_ctx, tr, w, F.FEW_FP64)
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    assert gm.shape[0] == 63115200
    mm_full = _mismatch_on_device(gm, g64)
    assert mm_full <= MIXED_MISMATCH, mm_full
    n = 100000
    i0 = w.n_samples - n
    o = _oracle(w, i0, n)
    assert oracle.mismatch(to_host(gm[i0:]), o) <= MIXED_MISMATCH
    assert rel_l2(to_host(g64[i0:]), o) <= FP64_REL_L2
    o2 = _oracle(w, 0, 2000)
    assert oracle.mismatch(to_host(gm[:2000]), o2) <= MIXED_MISMATCH
    assert rel_l2(to_host(g64[:2000]), o2) <= FP64_REL_L2
    del gm, g64
    tr.release()


TINY = [(1, 6, 1), (2, 7, 7), (3, 5, 255), (4, 9, 256), (5, 4, 257), (6, 12, 1023),
        (7, 8, 1025), (8, 30, 5000)]


@pytest.mark.parametrize("seed,K,ns", TINY)
def test_tiny_ragged(gpu_ctx, seed, K, ns):
    w = W.tiny_inputs(seed, K=K, n_samples=max(ns, 2))
    w.n_samples = ns
    o = _oracle(w)
    g = _gpu(gpu_ctx, w, F.FEW_FP64)
    assert rel_l2(g, o) <= FP64_REL_L2
    gm = _gpu(gpu_ctx, w, F.FEW_MIXED)
    assert oracle.mismatch(gm, o) <= MIXED_MISMATCH


@pytest.mark.parametrize("K", [180, 181, 4096])
def test_knot_counts_up_to_the_maximum(gpu_ctx, K):
    """Both forms of the spline build (values parked in shared memory up to K = 180, in the
    global scratch above) and the largest trajectory FEW_MAX_KNOTS = 4096, with a few samples
    per segment so that almost every pass is cut short by its segment's end."""
    w = W.tiny_inputs(900 + K, K=K, n_samples=5 * K)
    o = _oracle(w)
    g = _gpu(gpu_ctx, w, F.FEW_FP64)
    assert rel_l2(g, o) <= FP64_REL_L2, rel_l2(g, o)
    assert max_phase_err(g, o) <= FP64_PHASE
    gm = _gpu(gpu_ctx, w, F.FEW_MIXED)
    assert oracle.mismatch(gm, o) <= MIXED_MISMATCH


@pytest.mark.parametrize("K,ns", [(600, 50), (4096, 300), (40, 3)])
def test_segments_without_samples(gpu_ctx, K, ns):
    """Knots closer together than the sampling step: most segments hold no sample at all (their
    passes, anchors and folds must contribute nothing and write nothing)."""
    w = W.tiny_inputs(1200 + K, K=K, n_samples=ns, T=2.0e5, dt=2.0e5 / ns)
    seg = F.few_plan_segments(w.t_knots, w.t0, w.dt, w.n_samples)
    assert np.sum(np.diff(seg) == 0) > 0
    o = _oracle(w)
    g = _gpu(gpu_ctx, w, F.FEW_FP64)
    assert rel_l2(g, o) <= FP64_REL_L2, rel_l2(g, o)
    gm = _gpu(gpu_ctx, w, F.FEW_MIXED)
    assert oracle.mismatch(gm, o) <= MIXED_MISMATCH


MODESETS = {
    "single_22": [(2, 2, 0)],
    "m0_only": [(2, 0, -3), (2, 0, 3), (3, 0, 0), (4, 0, 1)],
    "odd_l": [(3, 1, 2), (3, 3, -4), (5, 2, 7), (7, 7, -1)],
    "wide_n": [(2, 2, -30), (2, 2, 30), (2, 1, 17), (10, 10, -25)],
    "high_l": [(12, 5, 3), (20, 20, -2), (32, 0, 1), (32, 31, 0)],
    # |n| at its limit: a row of 2049 slots streamed in many tiles, ~2000 powers of z_r in FP32
    "extreme_n": [(2, 2, -1024), (2, 2, 1024), (3, 1, 500), (2, 0, -700)],
}


@pytest.mark.parametrize("name", sorted(MODESETS))
def test_mode_sets(gpu_ctx, name):
    modes = np.asarray(MODESETS[name], dtype=np.int32)
    if name == "extreme_n":  # amplitudes that do not decay in n (FP32 range for the mixed path)
        w = W.make_inputs(2.0e5, 10, 2.0e5 / 3000, modes, 42, 8.0, 1.0e4, n_samples=3000)
    else:
        w = W.tiny_inputs(42, K=10, n_samples=3000, modes=modes)
    o = _oracle(w)
    g = _gpu(gpu_ctx, w, F.FEW_FP64)
    assert rel_l2(g, o) <= FP64_REL_L2, rel_l2(g, o)
    gm = _gpu(gpu_ctx, w, F.FEW_MIXED)
    assert oracle.mismatch(gm, o) <= MIXED_MISMATCH


@pytest.mark.parametrize("lmax,nmax", [(6, 80), (12, 80)])
def test_wide_mode_tables(gpu_ctx, lmax, nmax):
    """|n| up to 80: slot tables of 13 x 161 = 2093 and 25 x 161 = 4025 slots per segment, more
    than one shared-memory stage holds, streamed tile by tile (Sec. 3.C quotes 1e2-1e4 modes)."""
    modes = W.mode_grid(lmax, nmax)
    slots, rows = F.few_mode_slots(modes)
    assert slots == (2 * lmax + 1) * (2 * nmax + 1)
    # slow decay in l and n (sigma_l = 8, sigma_n = 60) so every slot carries weight
    w = W.make_inputs(2.0e5, 9, 2.0e5 / 1500, modes, 77 + lmax, 8.0, 60.0, n_samples=1500)
    o = _oracle(w)
    g = _gpu(gpu_ctx, w, F.FEW_FP64)
    assert rel_l2(g, o) <= FP64_REL_L2, rel_l2(g, o)
    assert max_phase_err(g, o) <= FP64_PHASE
    gm = _gpu(gpu_ctx, w, F.FEW_MIXED)
    assert oracle.mismatch(gm, o) <= MIXED_MISMATCH


def test_ragged_rows_with_shifts(gpu_ctx):
    """Rows whose lowest n differ (shifts between rows in both directions) and gaps in m."""
    modes = np.asarray([(2, 2, 5), (2, 2, 9), (3, 2, -4), (4, 1, 12), (4, 1, 13), (5, 5, -7),
                        (5, 0, -2), (6, 0, 3), (7, 3, 0), (9, 9, 1)], dtype=np.int32)
    w = W.tiny_inputs(5, K=8, n_samples=2500, modes=modes)
    o = _oracle(w)
    for S in (16, 512):
        saved = {p: gpu_ctx.get_tiles(p) for p in (F.FEW_FP64, F.FEW_MIXED)}
        try:
            for p, (R, T, _) in saved.items():
                gpu_ctx.set_tiles(p, R, T, S)
            g = _gpu(gpu_ctx, w, F.FEW_FP64)
            assert rel_l2(g, o) <= FP64_REL_L2, (S, rel_l2(g, o))
            gm = _gpu(gpu_ctx, w, F.FEW_MIXED)
            assert oracle.mismatch(gm, o) <= MIXED_MISMATCH
        finally:
            for p, tile in saved.items():
                gpu_ctx.set_tiles(p, *tile)


def test_offset_start_and_last_knot(gpu_ctx):
    """Samples from the middle of the trajectory up to exactly its last knot."""
    w = W.config1()
    dt = 7.0
    n = 20000
    t0 = w.t_knots[-1] - (n - 1) * dt
    w.t0, w.dt, w.n_samples = t0, dt, n
    o = _oracle(w)
    g = _gpu(gpu_ctx, w, F.FEW_FP64)
    assert rel_l2(g, o) <= FP64_REL_L2


def test_phase_offsets_and_scale(gpu_ctx):
    import torch
    w = W.config1()
    dpp, dpr, sc = 1.234, -2.5, 3.75
    tr = RT.from_inputs(gpu_ctx, w)
    out = RT.waveform(gpu_ctx, tr, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_FP64,
                      scale=sc, dphi_phi0=dpp, dphi_r0=dpr)
    torch.cuda.synchronize()
    g = to_host(out)
    tr.release()
    o = oracle.waveform(w.t_knots, w.phi_phi + dpp, w.phi_r + dpr, w.modes, w.amp_re, w.amp_im,
                        w.theta, w.phi, sc, w.t0, w.dt, 0, w.n_samples, oracle_threads())
    assert rel_l2(g, o) <= FP64_REL_L2


def test_host_buffers_match_device_path(gpu_ctx):
    import torch
    w = W.config1()
    g_dev = _gpu(gpu_ctx, w, F.FEW_FP64)
    tr = RT.from_inputs(gpu_ctx, w, device_data=False)
    host = np.zeros(w.n_samples, dtype=np.complex128)
    req = RT.request(tr, host, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_FP64,
                     out_where=F.FEW_MEM_HOST)
    F.few_waveform(gpu_ctx.handle, req, RT.current_stream())
    torch.cuda.synchronize()
    tr.release()
    np.testing.assert_array_equal(host, g_dev)


@pytest.mark.parametrize("pinned", [(1, 1, 1, 1), (0, 1, 1, 0), (1, 0, 0, 1)])
def test_pinned_host_inputs_match_device_inputs(gpu_ctx, pinned):
    """Knot arrays from page-locked and pageable host memory, in any mix, give the same spline
    data as device-resident ones, so the same output bits."""
    import torch
    w = W.config1()
    g_dev = _gpu(gpu_ctx, w, F.FEW_MIXED)
    arrays = (w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() if p
            else np.ascontiguousarray(a) for a, p in zip(arrays, pinned)]
    tr = RT.Trajectory(gpu_ctx, w.t_knots, w.modes)
    tr.set_data_host(*host)
    out = RT.waveform_inputs(gpu_ctx, tr, w, F.FEW_MIXED, None)
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    h = to_host(out)
    tr.release()
    np.testing.assert_array_equal(h, g_dev)


def test_pinned_host_output_matches_device_path(gpu_ctx):
    """Page-locked host output is stored directly by the summation kernel: same bits as a
    device-resident output, in both precisions."""
    import torch
    w = W.config1()
    tr = RT.from_inputs(gpu_ctx, w)
    for prec, dt in ((F.FEW_FP64, torch.complex128), (F.FEW_MIXED, torch.complex64)):
        dev = RT.alloc_out(w.n_samples, dt == torch.complex64)
        RT.waveform(gpu_ctx, tr, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec, scale=w.scale,
                    out=dev)
        host = torch.zeros(w.n_samples, dtype=dt).pin_memory().numpy()
        req = RT.request(tr, host, w.n_samples, w.t0, w.dt, w.theta, w.phi, prec, scale=w.scale,
                         out_where=F.FEW_MEM_HOST)
        F.few_waveform(gpu_ctx.handle, req, RT.current_stream())
        torch.cuda.synchronize()
        assert gpu_ctx.sync_status() == F.FEW_OK
        np.testing.assert_array_equal(host, dev.cpu().numpy())
    tr.release()


def test_tiles_are_bit_identical(gpu_ctx):
    """Every tile shape -- samples per thread, threads, slots per ring stage (including stages
    smaller than a row, so that rows straddle stages) -- gives the same bits: each sample is
    summed by one thread in a fixed order, and the mixed path's phase anchors sit at fixed
    sample indices."""
    w = W.config1()  # 9 rows of 11 slots
    ref = {}
    saved = {p: gpu_ctx.get_tiles(p) for p in (F.FEW_FP64, F.FEW_MIXED)}
    try:
        for prec, Rs in ((F.FEW_FP64, (1, 2)), (F.FEW_MIXED, (2, 4, 8))):
            for R in Rs:
                for T in (128, 256):
                    for S in (16, 48, 512):
                        gpu_ctx.set_tiles(prec, R, T, S)
                        g = _gpu(gpu_ctx, w, prec)
                        if prec not in ref:
                            ref[prec] = g
                        np.testing.assert_array_equal(g, ref[prec], err_msg=f"{prec} {R} {T} {S}")
    finally:
        for p, tile in saved.items():
            gpu_ctx.set_tiles(p, *tile)


def test_errors_and_noop(gpu_ctx):
    import torch
    w = W.tiny_inputs(3)
    tr = RT.Trajectory(gpu_ctx, w.t_knots, w.modes)
    out = RT.alloc_out(10, False)
    with pytest.raises(F.FewError) as e:  # no spline data yet
        F.few_waveform(gpu_ctx.handle, RT.request(tr, out, 10, 0.0, w.dt, 0.3, 0.2), 0)
    assert e.value.status == F.FEW_ERR_STATE
    tr.set_data_host(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
    with pytest.raises(F.FewError) as e:
        F.few_waveform(gpu_ctx.handle, RT.request(tr, out, 10, -1.0, w.dt, 0.3, 0.2), 0)
    assert e.value.status == F.FEW_ERR_RANGE
    with pytest.raises(F.FewError) as e:
        F.few_waveform(gpu_ctx.handle, RT.request(tr, out, 10, 0.0, w.T, 0.3, 0.2), 0)
    assert e.value.status == F.FEW_ERR_RANGE
    with pytest.raises(F.FewError) as e:
        F.few_waveform(gpu_ctx.handle, RT.request(tr, out, 10, 0.0, w.dt, float("nan"), 0.2), 0)
    assert e.value.status == F.FEW_ERR_INVALID_ARG
    # n_samples = 0 is a no-op
    F.few_waveform(gpu_ctx.handle, RT.request(tr, out, 0, 0.0, w.dt, 0.3, 0.2), 0)
    torch.cuda.synchronize()
    assert gpu_ctx.sync_status() == F.FEW_OK
    # a NaN in device-resident knot data is detected by the build kernel and latched
    bad = w.amp_re.copy()
    bad[2, 1] = np.nan
    tr.set_data_host(w.phi_phi, w.phi_r, bad, w.amp_im)
    assert gpu_ctx.sync_status() == F.FEW_ERR_INVALID_ARG
    assert gpu_ctx.sync_status() == F.FEW_OK  # latch cleared
    # infinities at the end rows (the first values each sweep loads) and a NaN in a phase
    K = w.phi_phi.shape[0]
    for which, row, col, val in [("amp_re", 0, 0, np.inf), ("amp_im", K - 1, 5, -np.inf),
                                 ("phi_r", K // 2, None, np.nan), ("phi_phi", K - 1, None, np.inf)]:
        arrs = {"phi_phi": w.phi_phi.copy(), "phi_r": w.phi_r.copy(),
                "amp_re": w.amp_re.copy(), "amp_im": w.amp_im.copy()}
        if col is None:
            arrs[which][row] = val
        else:
            arrs[which][row, col] = val
        tr.set_data_host(arrs["phi_phi"], arrs["phi_r"], arrs["amp_re"], arrs["amp_im"])
        assert gpu_ctx.sync_status() == F.FEW_ERR_INVALID_ARG, which
        assert gpu_ctx.sync_status() == F.FEW_OK
    tr.set_data_host(w.phi_phi, w.phi_r, w.amp_re, w.amp_im)
    assert gpu_ctx.sync_status() == F.FEW_OK
    tr.release()
    with pytest.raises(F.FewError) as e:
        RT.Trajectory(gpu_ctx, [0.0, 1.0, 2.0], w.modes)
    assert e.value.status == F.FEW_ERR_KNOTS


def test_budget_is_enforced():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = W.config1()
    with RT.Context(0, hbm_budget_bytes=1 << 20) as ctx:
        with pytest.raises(F.FewError) as e:
            RT.Trajectory(ctx, w.t_knots, W.mode_grid(10, 30))
        assert e.value.status == F.FEW_ERR_BUDGET
        used, budget = ctx.memory()
        assert used == 0 and budget == 1 << 20


def _gpu_phases(ctx, w, dpp=0.0, dpr=0.0):
    import torch
    tr = RT.from_inputs(ctx, w)
    buf = torch.empty(2 * w.n_samples, dtype=torch.float64, device="cuda")
    F.few_phase_samples(ctx.handle, tr.handle, w.t0, w.dt, w.n_samples, buf.data_ptr(), dpp, dpr,
                        RT.current_stream())
    torch.cuda.synchronize()
    tr.release()
    return buf.cpu().numpy().reshape(-1, 2)


@pytest.mark.parametrize("cfg", ["year", "four_year"])
def test_phase_step_matches_oracle(gpu_ctx, cfg):
    """Per-sample orbital phases (reduced, in turns) against the long-double oracle.

    Gate: every mode phase m*Phi_phi + n*Phi_r (|m| <= 10, |n| <= 30) within 1e-9 rad, i.e. each
    orbital phase within 1e-9/40 rad.
    """
    w = W.config2() if cfg == "year" else W.config5()
    g = _gpu_phases(gpu_ctx, w)
    worst = 0.0
    for i0 in (0, w.n_samples // 3, w.n_samples // 2 + 12345, w.n_samples - 3000):
        o = oracle.phases(w.t_knots, w.phi_phi, w.phi_r, w.t0, w.dt, i0, 3000)
        d = g[i0:i0 + 3000] - o
        d -= np.round(d)
        worst = max(worst, float(np.max(np.abs(d))) * 2 * math.pi)
    assert worst <= 1e-9 / 40, worst


def test_phase_step_offsets(gpu_ctx):
    w = W.config1()
    dpp, dpr = 1.0e3 + 0.25, -7.5
    g = _gpu_phases(gpu_ctx, w, dpp, dpr)
    o = oracle.phases(w.t_knots, w.phi_phi + dpp, w.phi_r + dpr, w.t0, w.dt, 0, w.n_samples)
    d = g - o
    d -= np.round(d)
    assert np.max(np.abs(d)) * 2 * math.pi <= 1e-9 / 40


@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
def test_detector_frame_output(gpu_ctx, prec):
    """Frame transformation (Sec. 2.A) fused into the harmonics: against the oracle's SSB sum."""
    import torch
    w = W.config1()
    tS, pS, tK, pK = 0.54, 5.36, 1.73, 3.20  # the angles of the paper's Sec. 6 study
    tr = RT.from_inputs(gpu_ctx, w)
    out = RT.alloc_out(w.n_samples, prec == F.FEW_MIXED)
    req = RT.request(tr, out, w.n_samples, w.t0, w.dt, tS, pS, prec, 1.0, frame=F.FEW_FRAME_SSB,
                     theta_K=tK, phi_K=pK)
    F.few_waveform(gpu_ctx.handle, req, RT.current_stream())
    torch.cuda.synchronize()
    g = to_host(out)
    o = oracle.waveform_ssb(w.t_knots, w.phi_phi, w.phi_r, w.modes, w.amp_re, w.amp_im, tS, pS,
                            tK, pK, 1.0, w.t0, w.dt, 0, w.n_samples, oracle_threads())
    if prec == F.FEW_FP64:
        assert rel_l2(g, o) <= FP64_REL_L2
    else:
        assert oracle.mismatch(g, o) <= MIXED_MISMATCH
    # R parallel to S has no source frame
    bad = RT.request(tr, out, 10, w.t0, w.dt, 0.3, 1.0, prec, frame=F.FEW_FRAME_SSB,
                     theta_K=0.3, phi_K=1.0)
    with pytest.raises(F.FewError):
        F.few_waveform(gpu_ctx.handle, bad, 0)
    tr.release()


def test_strongly_nonuniform_knots(gpu_ctx):
    """The spline build eliminates without pivoting from both ends of the reduced system; its
    diagonal dominance holds for any spacing, checked here on knot gaps that differ by 180x."""
    w = W.tiny_inputs(11, K=10, n_samples=4000)
    gaps = np.array([1.0, 1.0, 80.0, 0.5, 0.5, 90.0, 1.0, 60.0, 1.0])
    w.t_knots = np.r_[0.0, np.cumsum(gaps)] / gaps.sum() * w.t_knots[-1]
    w.phi_phi, w.phi_r = w.phases_at(w.t_knots)
    A = w.amp_model(w.t_knots)
    w.amp_re, w.amp_im = np.ascontiguousarray(A.real), np.ascontiguousarray(A.imag)
    o = _oracle(w)
    assert rel_l2(_gpu(gpu_ctx, w, F.FEW_FP64), o) <= FP64_REL_L2
    assert oracle.mismatch(_gpu(gpu_ctx, w, F.FEW_MIXED), o) <= MIXED_MISMATCH


def test_knot_count_limit(gpu_ctx):
    t = np.arange(4097, dtype=np.float64)  # one knot more than FEW_MAX_KNOTS
    with pytest.raises(F.FewError) as e:
        F.few_traj_create(gpu_ctx.handle, t, np.array([[2, 2, 0]], dtype=np.int32))
    assert e.value.status == F.FEW_ERR_LIMIT


def test_host_threads_in_flight(gpu_ctx):
    """Host threads calling few_traj_set_data / few_waveform with host buffers at once, each with
    its own trajectory, page-locked buffers and stream (the library releases the context while a
    call waits): every result equals the same waveform computed alone."""
    import threading
    import torch
    ws = [W.tiny_inputs(700 + k, K=12 + 5 * k, n_samples=20000 + 3001 * k) for k in range(3)]
    ref = [_gpu(gpu_ctx, w, F.FEW_MIXED) for w in ws]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    errs, results = [], [None] * len(ws)

    def worker(k):
        try:
            w = ws[k]
            tr = RT.Trajectory(gpu_ctx, w.t_knots, w.modes)
            h_in = [pin(a) for a in (w.phi_phi, w.phi_r, w.amp_re, w.amp_im)]
            out = torch.empty(w.n_samples, dtype=torch.complex64).pin_memory().numpy()
            req = RT.request(tr, out, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_MIXED,
                             scale=w.scale, out_where=F.FEW_MEM_HOST)
            s = torch.cuda.Stream()
            for _ in range(5):
                out[:] = 0
                F.few_traj_set_data(gpu_ctx.handle, tr.handle, *h_in, stream=int(s.cuda_stream))
                F.few_waveform(gpu_ctx.handle, req, int(s.cuda_stream))
                results[k] = out.copy()
                np.testing.assert_array_equal(results[k], ref[k])
            tr.release()
        except Exception as e:  # noqa: BLE001 -- re-raised below
            errs.append(e)
    ths = [threading.Thread(target=worker, args=(k,)) for k in range(len(ws))]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    if errs:
        raise errs[0]
    assert gpu_ctx.sync_status() == F.FEW_OK
