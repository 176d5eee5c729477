"""Pins for the oracle's frame transformation (Sec. 2.A).

* the source-frame azimuth of the propagation direction -R is -pi/2 for any geometry (the
  paper's statement), and cos(theta_src) = -R.S, both recomputed with numpy vectors;
* the polarization angle agrees with the vector form
  tan psi = (S.z - (S.R)(z.R)) / (R.(S x z)), compared through e^{2 i psi} (branch-free);
* the detector-frame waveform is -e^{-2 i psi} times the source-frame sum at those angles.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_04582_gb300 import workloads as W


def _unit(t, p):
    return np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])


@pytest.mark.parametrize("seed", range(8))
def test_angles_against_vector_geometry(seed):
    rng = np.random.default_rng(seed)
    tS, tK = np.arccos(rng.uniform(-1, 1, 2))
    pS, pK = rng.uniform(0, 2 * math.pi, 2)
    th, ph, psi = oracle.frame_angles(tS, pS, tK, pK)
    R, S = _unit(tS, pS), _unit(tK, pK)
    assert abs(ph + math.pi / 2) < 1e-12
    assert abs(math.cos(th) + R @ S) < 1e-12
    z = np.array([0.0, 0.0, 1.0])
    num = S @ z - (S @ R) * (z @ R)
    den = R @ np.cross(S, z)
    assert abs(np.exp(2j * psi) - np.exp(2j * math.atan2(num, den))) < 1e-12


def test_paper_angles():
    # the angles of the paper's mismatch study (Sec. 6)
    th, ph, psi = oracle.frame_angles(0.54, 5.36, 1.73, 3.20)
    R, S = _unit(0.54, 5.36), _unit(1.73, 3.20)
    assert abs(math.cos(th) + R @ S) < 1e-12 and abs(ph + math.pi / 2) < 1e-12


def test_parallel_vectors_are_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.frame_angles(0.3, 1.0, 0.3, 1.0)


def test_detector_frame_waveform_is_a_rotated_source_frame_sum():
    w = W.tiny_inputs(5)
    tS, pS, tK, pK = 0.54, 5.36, 1.73, 3.20
    th, ph, psi = oracle.frame_angles(tS, pS, tK, pK)
    src = oracle.waveform(w.t_knots, w.phi_phi, w.phi_r, w.modes, w.amp_re, w.amp_im, th, ph, 1.3,
                          w.t0, w.dt, 0, w.n_samples)
    ssb = oracle.waveform_ssb(w.t_knots, w.phi_phi, w.phi_r, w.modes, w.amp_re, w.amp_im, tS, pS,
                              tK, pK, 1.3, w.t0, w.dt, 0, w.n_samples)
    want = -np.exp(-2j * psi) * src
    assert np.max(np.abs(ssb - want)) < 1e-14 * np.max(np.abs(want))
