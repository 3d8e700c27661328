"""Penalised IMEX step (oracle): the alternative to the exponential method that
Section 4 names, where the anisotropic diffusion is penalised by an isotropic
operator treated implicitly and the rest is treated explicitly.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline, never by the product path.

The paper gives no formula (it cites its companion work).  Readings (listed
in the design notes):
  * penalty operator P = beta L, with L the operator of Eq. anidiff for the
    unit isotropic tensor (D = I, a = 0) on the same grid and boundary
    condition (the 5-point Laplacian of the flux form);
  * beta = max over cells of the largest eigenvalue of D unless given (the
    penalised scheme is stable for beta >= lambda_max(D) / 2; the factor 2
    is a safety margin);
  * first-order IMEX Euler: the penalty implicit, everything else explicit,
        (I - dt P) u+ = u + dt ((A - P) u + S(t)),
    solved as (I - dt P) delta = dt (A u + S(t)), u+ = u + delta.

Pins (tests/test_oracle_penalised.py): beta = 0 is the explicit Euler step,
first-order convergence to the exact solution (dense exponential), bounded
solutions at step sizes far beyond the explicit limit, and the exact
solution of the implicit system.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operator import assemble


def penalty_operator(grid) -> sp.csr_matrix:
    """L: the operator of Eq. anidiff with D = I and a = 0."""
    return assemble(grid, 1.0, 0.0, 1.0)


def default_beta(Dxx, Dxy, Dyy) -> float:
    """max over cells of lambda_max(D)."""
    Dxx, Dxy, Dyy = (np.asarray(a, dtype=np.float64) for a in (Dxx, Dxy, Dyy))
    tr = 0.5 * (Dxx + Dyy)
    return float(np.max(tr + np.sqrt(0.25 * (Dxx - Dyy) ** 2 + Dxy ** 2)))


def imex_step(A, L, u, t, dt, source_at, beta):
    """One penalised IMEX Euler step; returns u+ (exact sparse solve)."""
    u = np.asarray(u, dtype=np.float64)
    rhs = dt * (A @ u + source_at(t))
    M = sp.identity(A.shape[0], format="csc") - (dt * beta) * L.tocsc()
    delta = spla.spsolve(M, rhs)
    return u + delta
