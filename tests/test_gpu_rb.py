"""Mode amplitudes from reduced-basis coefficients (Sec. 3.E) on the GPU against the oracle:
the FP64 GEMM and the tensor-core (split bf16, FP32 accumulation) product, with and without
the per-knot renormalisation, at the paper's size (99 coefficients, 3843 modes) and at ragged
sizes that leave partial tiles in every dimension; then the amplitudes feed a trajectory and
its waveform is compared with the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import fewsum as F
from paper_2104_04582_gb300 import runtime as RT
from paper_2104_04582_gb300 import workloads as W
from tests.gpu_common import MIXED_MISMATCH, oracle_threads, to_host

pytestmark = pytest.mark.gpu

# Per-row bounds in the form of the dot-product error bound |fl(x.y) - x.y| <= g |x|.|y|:
# FP64, a 2 Nb-term complex dot product per output; mixed, FP32 accumulation of six partial
# products of bf16 parts (the three-way split keeps ~24 bits of each operand) over 12 Nb terms,
# so g = 2e-6 (about 32 FP32 ulps, the typical sqrt(12 Nb) growth with margin).
FP64_GAMMA = 1e-14
MIXED_GAMMA = 2e-6


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _gpu_rb(ctx, alpha, basis, norms, prec, basis_on_device=False):
    import torch
    M, N = alpha.shape[0], basis.shape[1]
    if basis_on_device:
        h = F.few_basis_create(ctx.handle, _dev(basis.real), _dev(basis.imag), RT.current_stream())
    else:
        h = F.few_basis_create(ctx.handle, basis.real, basis.imag, RT.current_stream())
    try:
        ore = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
        oim = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
        F.few_rb_amplitudes(ctx.handle, h, _dev(alpha.real), _dev(alpha.imag), ore, oim,
                            None if norms is None else _dev(norms), prec, RT.current_stream())
        torch.cuda.synchronize()
        assert ctx.sync_status() == F.FEW_OK
        return to_host(ore) + 1j * to_host(oim)
    finally:
        F.few_basis_release(ctx.handle, h)


def _check_rows(g, o, alpha, basis, norms, prec):
    """||g_k - o_k|| <= gamma || |s_k alpha_k| |B| || for every knot k."""
    raw = np.abs(alpha) @ np.abs(basis)
    if norms is not None:
        plain = np.linalg.norm(oracle.rb_amplitudes(alpha, basis), axis=1)
        s = np.where(plain > 0, norms / np.where(plain > 0, plain, 1.0), 0.0)
        raw = raw * s[:, None]
    gamma = FP64_GAMMA if prec == F.FEW_FP64 else MIXED_GAMMA
    err = np.linalg.norm(g - o, axis=1)
    bound = gamma * np.linalg.norm(raw, axis=1)
    assert np.all(err <= bound), np.max(err / np.where(bound > 0, bound, 1e-300))


@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
@pytest.mark.parametrize("renorm", [False, True])
def test_rb_paper_size_matches_oracle(gpu_ctx, prec, renorm):
    alpha, basis, nu = W.rb_inputs(100)
    g = _gpu_rb(gpu_ctx, alpha, basis, nu if renorm else None, prec)
    o = oracle.rb_amplitudes(alpha, basis, nu if renorm else None, oracle_threads())
    assert np.all(np.isfinite(g))
    _check_rows(g, o, alpha, basis, nu if renorm else None, prec)


@pytest.mark.parametrize("M,Nb,N", [(1, 1, 1), (129, 7, 130), (300, 99, 257), (5, 256, 64),
                                    (257, 33, 1)])
@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
def test_rb_ragged_sizes(gpu_ctx, M, Nb, N, prec):
    rng = np.random.default_rng(M * 1000 + Nb * 10 + N)
    alpha = rng.standard_normal((M, Nb)) + 1j * rng.standard_normal((M, Nb))
    basis = rng.standard_normal((Nb, N)) + 1j * rng.standard_normal((Nb, N))
    nu = rng.uniform(0.5, 2.0, M)
    g = _gpu_rb(gpu_ctx, alpha, basis, nu, prec, basis_on_device=(M % 2 == 1))
    o = oracle.rb_amplitudes(alpha, basis, nu)
    _check_rows(g, o, alpha, basis, nu, prec)


@pytest.mark.parametrize("prec", [F.FEW_FP64, F.FEW_MIXED])
def test_rb_norms_and_zero_rows(gpu_ctx, prec):
    alpha, basis, nu = W.rb_inputs(40, Nb=20, N=500)
    alpha[[3, 17]] = 0.0
    g = _gpu_rb(gpu_ctx, alpha, basis, nu, prec)
    norms = np.linalg.norm(g, axis=1)
    live = np.ones(40, bool)
    live[[3, 17]] = False
    tol = 1e-13 if prec == F.FEW_FP64 else 3e-6
    assert np.all(np.abs(norms[live] - nu[live]) <= tol * nu[live])
    assert np.all(g[~live] == 0)


def test_rb_bad_norm_latches_invalid(gpu_ctx):
    import torch
    alpha, basis, nu = W.rb_inputs(8, Nb=4, N=16)
    nu[5] = np.nan
    nu[6] = -1.0
    h = F.few_basis_create(gpu_ctx.handle, basis.real, basis.imag, RT.current_stream())
    try:
        ore = torch.empty((8, 16), dtype=torch.float64, device="cuda")
        oim = torch.empty_like(ore)
        F.few_rb_amplitudes(gpu_ctx.handle, h, _dev(alpha.real), _dev(alpha.imag), ore, oim,
                            _dev(nu), F.FEW_MIXED, RT.current_stream())
        torch.cuda.synchronize()
        assert gpu_ctx.sync_status() == F.FEW_ERR_INVALID_ARG
        assert gpu_ctx.sync_status() == F.FEW_OK  # the latch is cleared once read
    finally:
        F.few_basis_release(gpu_ctx.handle, h)


def test_rb_zero_knots_is_noop(gpu_ctx):
    import torch
    alpha, basis, _ = W.rb_inputs(4, Nb=3, N=8)
    h = F.few_basis_create(gpu_ctx.handle, basis.real, basis.imag, RT.current_stream())
    try:
        e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
        o = torch.empty((0, 8), dtype=torch.float64, device="cuda")
        F.few_rb_amplitudes(gpu_ctx.handle, h, e, e, o, o, None, F.FEW_MIXED, RT.current_stream())
        torch.cuda.synchronize()
        assert gpu_ctx.sync_status() == F.FEW_OK
    finally:
        F.few_basis_release(gpu_ctx.handle, h)


def test_rb_amplitudes_feed_a_waveform(gpu_ctx):
    """Amplitudes produced on the device straight into the arrays a trajectory reads, then the
    interpolated summation, against the oracle waveform built from the oracle's amplitudes."""
    import torch
    w = W.config1()  # one week, 40 knots, 132 modes
    K, N = len(w.t_knots), len(w.modes)
    alpha, basis, nu = W.rb_inputs(K, Nb=12, N=N)
    h = F.few_basis_create(gpu_ctx.handle, basis.real, basis.imag, RT.current_stream())
    tr = RT.Trajectory(gpu_ctx, w.t_knots, w.modes)
    try:
        ore = torch.empty((K, N), dtype=torch.float64, device="cuda")
        oim = torch.empty_like(ore)
        F.few_rb_amplitudes(gpu_ctx.handle, h, _dev(alpha.real), _dev(alpha.imag), ore, oim,
                            _dev(nu), F.FEW_MIXED, RT.current_stream())
        tr.set_data_device((_dev(w.phi_phi), _dev(w.phi_r), ore, oim))
        out = RT.waveform(gpu_ctx, tr, w.n_samples, w.t0, w.dt, w.theta, w.phi, F.FEW_MIXED,
                          scale=w.scale)
        torch.cuda.synchronize()
        assert gpu_ctx.sync_status() == F.FEW_OK
        A = oracle.rb_amplitudes(alpha, basis, nu)
        ref = oracle.waveform(w.t_knots, w.phi_phi, w.phi_r, w.modes, A.real, A.imag, w.theta,
                              w.phi, w.scale, w.t0, w.dt, 0, w.n_samples, oracle_threads())
        assert oracle.mismatch(to_host(out), ref) <= MIXED_MISMATCH
    finally:
        tr.release()
        F.few_basis_release(gpu_ctx.handle, h)


def test_rb_basis_limit(gpu_ctx):
    b = np.zeros((257, 4))  # one more basis vector than FEW_MAX_BASIS
    with pytest.raises(F.FewError) as e:
        F.few_basis_create(gpu_ctx.handle, b, b)
    assert e.value.status == F.FEW_ERR_LIMIT
