"""Spectral bounds of A (oracle), Section 2 of the paper.

The paper estimates the largest-magnitude eigenvalue alpha by Gershgorin's
disc theorem and takes the smallest as 0 (Section 2).  A power-iteration
estimate is offered as the tighter alternative.

Pins (tests/test_oracle_spectral.py): Gershgorin bound below every eigenvalue
of dense A for small grids; the constant-coefficient periodic case against the
hand-computed row sum; power iteration against the extreme eigenvalue of a
symmetric A (a = 0) from LAPACK.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

MASK64 = (1 << 64) - 1


def gershgorin(A: sp.csr_matrix) -> float:
    """alpha = min_i (a_ii - sum_{j != i} |a_ij|), a lower bound of Re(lambda)."""
    A = sp.csr_matrix(A)
    diag = A.diagonal()
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    return float(np.min(diag - (absrow - np.abs(diag))))


def splitmix64_uniform(n: int, seed: int) -> np.ndarray:
    """Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014; Vigna's
    reference form): output k mixes state = seed + (k+1) * 0x9E3779B97F4A7C15.
    Returns doubles in [-0.5, 0.5): (z >> 11) * 2^-53 - 0.5."""
    out = np.empty(n, dtype=np.float64)
    golden = 0x9E3779B97F4A7C15
    for k in range(n):
        z = (seed + (k + 1) * golden) & MASK64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        z = z ^ (z >> 31)
        out[k] = (z >> 11) * (2.0 ** -53) - 0.5
    return out


def power_iteration(A, x0, iters: int = 30, safety: float = 1.1):
    """Estimate |lambda|_max by normalised power iteration and return
    (alpha, estimate) with alpha = -safety * estimate.

    x <- x0 / ||x0||; repeat ``iters`` times: y = A x, est = ||y||, x = y / est.
    """
    x = np.asarray(x0, dtype=np.float64)
    x = x / np.linalg.norm(x)
    est = 0.0
    for _ in range(iters):
        y = A @ x
        est = float(np.linalg.norm(y))
        if est == 0.0:
            break
        x = y / est
    return -safety * est, est
