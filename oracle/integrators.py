"""Exponential quadrature time steps (oracle), Section 2 of the paper.

Eq. exp_quad:     u+ = u + dt sum_i b_i(dt A)(A u + S(t + c_i dt))
weights:          s = 1: b_1 = phi_1;
                  s = 2: b_1 = (c_2 phi_1 - phi_2)/(c_2 - c_1),
                         b_2 = (-c_1 phi_1 + phi_2)/(c_2 - c_1).
Eq. exp_midpoint: s = 1, c_1 = 1/2.
Eq. exp_quad_Gauss: s = 2, c = (1 -+ 1/sqrt 3)/2.

For s = 2 the sum of phi terms is collected (algebra only) as
    u+ = u + dt phi_1(dt A) w1 + dt^2 phi_2(dt A) w2,
    w1 = A u + (c_2 S_1 - c_1 S_2)/(c_2 - c_1),  w2 = (S_2 - S_1)/((c_2 - c_1) dt),
and evaluated as the exponential of the augmented matrix (Section 2, citing
Sidje98).  For s = 1 the phi_1 series is applied directly.

Pins (tests/test_oracle_integrators.py): dense expm/eigendecomposition
references, exactness of the midpoint rule for a time-independent source, mass
conservation, Fourier-mode decay and the temporal orders 2 and 4.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

from .leja import MAX_ITERS, LejaStats, leja_exp_augmented, leja_phi1


def expquad_step(A, u, t, dt, s, c: Sequence[float], source_at: Callable[[float], np.ndarray],
                 alpha, tol=1e-10, force_iters=None, rho_max=200.0, max_iters=MAX_ITERS,
                 adaptive=False):
    """One step of Eq. exp_quad with s in {1, 2}.  Returns (u+, LejaStats).
    adaptive: the adaptive substep control of oracle.leja (u is returned
    unchanged if it gives up)."""
    u = np.asarray(u, dtype=np.float64)
    Au = A @ u
    if s == 1:
        v = Au + source_at(t + c[0] * dt)
        q, st = leja_phi1(A, v, dt, alpha, tol, force_iters, rho_max, max_iters, adaptive)
        st.matvecs += 1
        if not st.converged and adaptive:
            return u.copy(), st
        return u + dt * q, st
    if s != 2:
        raise ValueError("s must be 1 or 2")
    c1, c2 = float(c[0]), float(c[1])
    S1 = source_at(t + c1 * dt)
    S2 = source_at(t + c2 * dt)
    w1 = Au + (c2 * S1 - c1 * S2) / (c2 - c1)
    w2 = (S2 - S1) / ((c2 - c1) * dt)
    top, _, st = leja_exp_augmented(A, np.zeros_like(u), np.array([0.0, 1.0]), w1, w2, dt,
                                    alpha, tol, force_iters, rho_max, max_iters, adaptive)
    st.matvecs += 1
    if not st.converged and adaptive:
        return u.copy(), st
    return u + top, st


def run(A, u0, t0, dt, steps, s, c, source_at, alpha, tol=1e-10, rho_max=200.0):
    """``steps`` consecutive steps; returns (u, list of LejaStats)."""
    u, t, stats = np.asarray(u0, dtype=np.float64), t0, []
    for _ in range(steps):
        u, st = expquad_step(A, u, t, dt, s, c, source_at, alpha, tol, None, rho_max)
        stats.append(st)
        t += dt
    return u, stats
