"""Seeded synthetic inputs for the interpolated mode summation.

This module defines *workloads*, not the method: it produces sparse trajectory knots
(times, the two orbital phases, and every mode's complex amplitude at the knots), the
mode list, viewing angles and the dense sampling grid.  Both the CUDA path and the CPU
oracle consume these arrays; neither computes anything here.

The paper's own inputs come from its flux-driven trajectory and its amplitude network
(Sec. 3.A-3.B, Sec. 4), neither of which is available, so synthetic stand-ins with the
same shapes are used:

* ~100 sparse knots per trajectory (Sec. 3.A), denser toward the plunge;
* one year at 0.1 Hz is ~3.15e6 samples (Sec. 3.C); LISA-like 10 s cadence (Sec. 6);
* the Schwarzschild eccentric mode grid l in [2,10], m in [0,l], n in [-30,30], i.e.
  3843 modes with m >= 0 (Sec. 4.B), m < 0 supplied by the symmetry of Eq. (amp_symmetry);
* epsilon-style mode subsets chosen by a cumulative-power threshold (Sec. 3.D, Sec. 6.A).

Phase model: Omega_phi(t) = 2*pi*5e-4*(1 - t/t_p)^(-3/8) rad/s, Omega_r = kappa(t)*Omega_phi
with kappa rising linearly 0.80 -> 0.95 over the duration T, t_p = 1.5*T; the phases are
the closed-form integrals of these (Sec. 2, phase integrals) plus uniform initial phases.
Amplitudes: A_lmn(t) = a_lmn*(1 + alpha*t/T + beta*(t/T)^2)*exp(i*psi).

Every generator takes an explicit seed and uses one numpy Generator(PCG64).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

YEAR_S = 365.25 * 86400.0
WEEK_S = 7.0 * 86400.0

OMEGA0 = 2.0 * math.pi * 5e-4  # rad/s, azimuthal frequency scale of the synthetic inspiral
KAPPA0, KAPPA1 = 0.80, 0.95     # Omega_r / Omega_phi at t = 0 and t = T


# --------------------------------------------------------------------------- grids

def knot_times(T: float, K: int) -> np.ndarray:
    """Knots t_k = T*(1 - (1 - k/(K-1))^2): spacing shrinks linearly toward T."""
    if K < 2:
        raise ValueError("K >= 2")
    k = np.arange(K, dtype=np.float64)
    t = T * (1.0 - (1.0 - k / (K - 1)) ** 2)
    t[0] = 0.0
    t[-1] = T
    return t


def n_samples_for(T: float, dt: float) -> int:
    """floor(T/dt) samples at t_i = i*dt, all inside [0, T]."""
    return int(math.floor(T / dt + 1e-9))


def mode_grid(lmax: int = 10, nmax: int = 30, lmin: int = 2) -> np.ndarray:
    """All (l, m, n) with lmin<=l<=lmax, 0<=m<=l, -nmax<=n<=nmax; int32 [N, 3]."""
    out = [(l, m, n) for l in range(lmin, lmax + 1) for m in range(0, l + 1)
           for n in range(-nmax, nmax + 1)]
    return np.asarray(out, dtype=np.int32).reshape(-1, 3)


# --------------------------------------------------------------------------- phases

def phase_phi(t: np.ndarray, T: float, phi0: float, tp: Optional[float] = None) -> np.ndarray:
    """Closed-form integral of Omega_phi from 0 to t (rad), plus phi0."""
    tp = 1.5 * T if tp is None else tp
    u = 1.0 - np.asarray(t, dtype=np.float64) / tp
    return phi0 + OMEGA0 * tp * (8.0 / 5.0) * (1.0 - u ** 0.625)


def phase_r(t: np.ndarray, T: float, phi0: float, tp: Optional[float] = None) -> np.ndarray:
    """Closed-form integral of kappa(t)*Omega_phi from 0 to t (rad), plus phi0.

    With u = 1 - t/t_p and kappa = a + b*(1-u), a = KAPPA0, b = (KAPPA1-KAPPA0)*t_p/T.
    """
    tp = 1.5 * T if tp is None else tp
    u = 1.0 - np.asarray(t, dtype=np.float64) / tp
    a = KAPPA0
    b = (KAPPA1 - KAPPA0) * tp / T
    return phi0 + OMEGA0 * tp * ((a + b) * (8.0 / 5.0) * (1.0 - u ** 0.625)
                                 - b * (8.0 / 13.0) * (1.0 - u ** 1.625))


# --------------------------------------------------------------------------- amplitudes

@dataclasses.dataclass
class AmpModel:
    """A_lmn(t) = a*(1 + alpha*t/T + beta*(t/T)^2)*exp(i*psi), per mode."""
    a: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    psi: np.ndarray
    T: float

    def __call__(self, t: np.ndarray) -> np.ndarray:
        """Complex [len(t), N] closed-form amplitudes."""
        x = np.asarray(t, dtype=np.float64)[:, None] / self.T
        env = self.a[None, :] * (1.0 + self.alpha[None, :] * x + self.beta[None, :] * x * x)
        return env * np.exp(1j * self.psi)[None, :]


def amp_scales(modes: np.ndarray, rng: np.random.Generator, sigma_l: float = 1.0,
               sigma_n: float = 3.0) -> np.ndarray:
    """a_lmn = 10^(-(l-2)/sigma_l) * exp(-|n-1|/sigma_n) * lognormal(0, 0.3)."""
    l = modes[:, 0].astype(np.float64)
    n = modes[:, 2].astype(np.float64)
    return (10.0 ** (-(l - 2.0) / sigma_l) * np.exp(-np.abs(n - 1.0) / sigma_n)
            * rng.lognormal(0.0, 0.3, size=len(modes)))


def select_by_power(modes: np.ndarray, a: np.ndarray, eps: float = 1e-5,
                    nmin: int = 10, nmax: int = 3843) -> np.ndarray:
    """Indices of the modes kept by a cumulative-power rule.

    Sort |a|^2 descending (ties by list index), keep until the running sum reaches
    (1-eps) of the total, then clamp the count to [nmin, nmax].  Returned indices are in
    the original list order.
    """
    p = np.abs(a) ** 2
    order = np.lexsort((np.arange(len(p)), -p))
    c = np.cumsum(p[order])
    keep = int(np.searchsorted(c, (1.0 - eps) * c[-1]) + 1)
    keep = max(nmin, min(nmax, keep, len(p)))
    return np.sort(order[:keep])


# --------------------------------------------------------------------------- inputs

@dataclasses.dataclass
class WaveformInputs:
    """Everything one waveform request needs (host numpy arrays)."""
    name: str
    T: float
    t_knots: np.ndarray      # f64 [K]
    phi_phi: np.ndarray      # f64 [K], rad
    phi_r: np.ndarray        # f64 [K], rad
    modes: np.ndarray        # i32 [N, 3] (l, m >= 0, n)
    amp_re: np.ndarray       # f64 [K, N]
    amp_im: np.ndarray       # f64 [K, N]
    theta: float
    phi: float
    t0: float
    dt: float
    n_samples: int
    scale: float = 1.0
    phi_phi0: float = 0.0
    phi_r0: float = 0.0
    amp_model: Optional[AmpModel] = None

    @property
    def K(self) -> int:
        return int(self.t_knots.shape[0])

    @property
    def N(self) -> int:
        return int(self.modes.shape[0])

    def mode_samples(self) -> int:
        return self.N * self.n_samples

    def phases_at(self, t: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
        """Closed-form phases of the synthetic inspiral at arbitrary times."""
        return (phase_phi(t, self.T, self.phi_phi0), phase_r(t, self.T, self.phi_r0))


def make_inputs(T: float, K: int, dt: float, modes: np.ndarray, seed: int,
                sigma_l: float = 1.0, sigma_n: float = 3.0, name: str = "custom",
                n_samples: Optional[int] = None) -> WaveformInputs:
    """Synthetic trajectory + amplitudes at the knots, with fixed seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = knot_times(T, K)
    phi_phi0 = float(rng.uniform(0.0, 2.0 * math.pi))
    phi_r0 = float(rng.uniform(0.0, 2.0 * math.pi))
    modes = np.ascontiguousarray(modes, dtype=np.int32)
    N = modes.shape[0]
    a = amp_scales(modes, rng, sigma_l, sigma_n)
    alpha = rng.uniform(-0.5, 0.5, size=N)
    beta = rng.uniform(-0.5, 0.5, size=N)
    psi = rng.uniform(0.0, 2.0 * math.pi, size=N)
    model = AmpModel(a, alpha, beta, psi, T)
    A = model(t)
    theta = float(np.arccos(rng.uniform(-1.0, 1.0)))
    phi = float(rng.uniform(0.0, 2.0 * math.pi))
    ns = n_samples_for(T, dt) if n_samples is None else int(n_samples)
    return WaveformInputs(
        name=name, T=T, t_knots=t,
        phi_phi=phase_phi(t, T, phi_phi0), phi_r=phase_r(t, T, phi_r0),
        modes=modes, amp_re=np.ascontiguousarray(A.real), amp_im=np.ascontiguousarray(A.imag),
        theta=theta, phi=phi, t0=0.0, dt=dt, n_samples=ns,
        phi_phi0=phi_phi0, phi_r0=phi_r0, amp_model=model)


# Named workloads (durations, cadences, knot counts and mode sets of the paper's runs).
SEEDS = {"C1": 20210409, "C2": 20210410, "C3": 20210411, "C4": 20210412, "C5": 20210413}


def config1(seed: int = SEEDS["C1"]) -> WaveformInputs:
    """One week at dt = 10 s (60,480 samples), K = 40, l=2..4, n=-5..5 (132 modes)."""
    return make_inputs(WEEK_S, 40, 10.0, mode_grid(4, 5), seed, name="C1: 1 week, 132 modes")


def config2(seed: int = SEEDS["C2"]) -> WaveformInputs:
    """One year at dt = 10 s (3,155,760 samples), K = 100, full 3843-mode grid."""
    return make_inputs(YEAR_S, 100, 10.0, mode_grid(10, 30), seed,
                       name="C2: 1 yr, dt=10 s, 3843 modes")


def config5(seed: int = SEEDS["C5"]) -> WaveformInputs:
    """Four years at dt = 2 s (63,115,200 samples), K = 300, full 3843-mode grid."""
    return make_inputs(4.0 * YEAR_S, 300, 2.0, mode_grid(10, 30), seed,
                       name="C5: 4 yr, dt=2 s, 3843 modes")


def _log_uniform(rng: np.random.Generator, lo: float, hi: float) -> float:
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def subset_waveform(rng: np.random.Generator, T: float, K: int, dt: float,
                    nmax_modes: int, name: str) -> WaveformInputs:
    """A waveform whose modes are the power-selected subset of the full grid.

    Each waveform draws its own amplitude decay scales sigma_l ~ logU(0.5, 8) and
    sigma_n ~ logU(1, 60), so the selected mode count spans the 10..3843 range.
    """
    grid = mode_grid(10, 30)
    sigma_l = _log_uniform(rng, 0.5, 8.0)
    sigma_n = _log_uniform(rng, 1.0, 60.0)
    seed = int(rng.integers(0, 2 ** 62))
    full = make_inputs(T, K, dt, grid, seed, sigma_l, sigma_n, name=name)
    keep = select_by_power(grid, full.amp_model.a, 1e-5, 10, nmax_modes)
    m = full.amp_model
    sub_model = AmpModel(m.a[keep], m.alpha[keep], m.beta[keep], m.psi[keep], T)
    full.modes = np.ascontiguousarray(grid[keep])
    full.amp_re = np.ascontiguousarray(full.amp_re[:, keep])
    full.amp_im = np.ascontiguousarray(full.amp_im[:, keep])
    full.amp_model = sub_model
    return full


def config3(n_waveforms: int = 256, seed: int = SEEDS["C3"]) -> List[WaveformInputs]:
    """Batch: T ~ U(0.25, 2) yr at dt = 10 s, K ~ U{50..150}, power-selected modes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for w in range(n_waveforms):
        T = float(rng.uniform(0.25, 2.0)) * YEAR_S
        K = int(rng.integers(50, 151))
        out.append(subset_waveform(rng, T, K, 10.0, 3843, name=f"C3[{w}]"))
    return out


@dataclasses.dataclass
class ServingRequest:
    """One request of the MCMC-like stream: a trajectory key plus per-request parameters."""
    arrival_s: float
    traj_key: int
    theta: float
    phi: float
    scale: float
    dphi_phi0: float
    dphi_r0: float
    dt: float
    T: float


def config4_stream(n_requests: int, rate_hz: float, seed: int = SEEDS["C4"],
                   p_new: float = 0.1) -> Tuple[Dict[int, WaveformInputs], List[ServingRequest]]:
    """Poisson arrivals; each request perturbs a resident trajectory or (p_new) a new one.

    Trajectories: T ~ U(0.5, 4) yr, dt in {5, 10, 15} s, K ~ U{50..150}, 10..1000 modes.
    Returns the trajectory table (key -> inputs) and the request list.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    trajs: Dict[int, WaveformInputs] = {}
    reqs: List[ServingRequest] = []
    t = 0.0
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        if not trajs or rng.uniform() < p_new:
            key = len(trajs)
            T = float(rng.uniform(0.5, 4.0)) * YEAR_S
            K = int(rng.integers(50, 151))
            dt = float(rng.choice([5.0, 10.0, 15.0]))
            trajs[key] = subset_waveform(rng, T, K, dt, 1000, name=f"C4 traj {key}")
        else:
            key = int(rng.integers(0, len(trajs)))
        base = trajs[key]
        reqs.append(ServingRequest(
            arrival_s=t, traj_key=key,
            theta=float(np.arccos(rng.uniform(-1.0, 1.0))),
            phi=float(rng.uniform(0.0, 2.0 * math.pi)),
            scale=float(rng.uniform(0.5, 2.0)),
            dphi_phi0=float(rng.normal(0.0, 0.1)), dphi_r0=float(rng.normal(0.0, 0.1)),
            dt=base.dt, T=base.T))
    return trajs, reqs


def tiny_inputs(seed: int, K: int = 6, n_samples: int = 200, modes: Optional[np.ndarray] = None,
                T: float = 2.0e5, dt: Optional[float] = None) -> WaveformInputs:
    """Small random case for brute-force checks (few knots, few modes, few samples)."""
    if modes is None:
        modes = np.asarray([(2, 2, 0), (2, 1, 1), (2, 0, -1), (3, 3, 2), (3, 0, 1),
                            (3, 2, -2), (4, 4, -1), (4, 1, 0)], dtype=np.int32)
    if dt is None:
        dt = T / n_samples
    return make_inputs(T, K, dt, modes, seed, name="tiny", n_samples=n_samples)


SEEDS["RB"] = 20210414


def rb_inputs(M: int, Nb: int = 99, N: int = 3843, seed: int = SEEDS["RB"], n_traj: int = 1):
    """Reduced-basis amplitude inputs (Sec. 3.E shapes: 99 complex coefficients per knot, 3843
    modes).  The basis has orthonormal rows (a greedy reduced basis is orthonormalised as it is
    built); coefficient j has weight exp(-j/20) (the decay of a reduced basis' projections) and
    drifts smoothly along each of `n_traj` trajectories of M / n_traj knots; the target norms
    are the coefficient norms times 1 + 1e-3 sin(...), standing in for the fit error between
    the network output and the trajectory's norm spline.
    Returns (alpha [M, Nb] complex, basis [Nb, N] complex, norms [M])."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((N, Nb)) + 1j * rng.standard_normal((N, Nb))
    q, _ = np.linalg.qr(g)
    basis = np.ascontiguousarray(q.T)
    w = np.exp(-np.arange(Nb) / 20.0)
    per = max(1, -(-M // n_traj))
    x = (np.arange(M) % per) / max(per - 1, 1)  # position along each trajectory, 0..1
    ph0 = rng.uniform(0.0, 2.0 * math.pi, Nb)
    rate = rng.uniform(0.5, 3.0, Nb)
    traj = np.arange(M) // per
    off = rng.uniform(0.0, 2.0 * math.pi, (n_traj, Nb))[traj]
    alpha = w * (1.0 + 0.3 * np.sin(2 * math.pi * rate * x[:, None] + off)) \
        * np.exp(1j * (ph0 + 4.0 * rate * x[:, None]))
    norms = np.linalg.norm(alpha, axis=1) * (1.0 + 1e-3 * np.sin(7.0 * x + traj))
    return np.ascontiguousarray(alpha), basis, norms
