"""Helpers shared by the GPU test modules (metrics and fixtures; no method arithmetic)."""
import os

import numpy as np
import pytest

# Gates (from the precision contract of the two paths):
#   FP64 path: relative L2 error <= 1e-10 and max phase error <= 1e-9 rad against the oracle;
#   mixed path: mismatch <= 1e-6 against the FP64 oracle.
FP64_REL_L2 = 1e-10
FP64_PHASE = 1e-9
MIXED_MISMATCH = 1e-6
# Phase error is measured where |h| >= PHASE_FLOOR * max|h| (arg is ill-conditioned near 0).
PHASE_FLOOR = 1e-3


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_phase_err(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    mask = np.abs(b) >= PHASE_FLOOR * np.max(np.abs(b))
    return float(np.max(np.abs(np.angle(a[mask] / b[mask]))))


def oracle_threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def to_host(t) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.complex128)
