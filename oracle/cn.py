"""Crank-Nicolson with restarted GMRES (oracle): the paper's comparison solver.

The paper compares against Crank-Nicolson (abstract; Section 3) but states
neither its source treatment nor its linear solver.  Reading used here:
    (I - dt/2 A) u+ = (I + dt/2 A) u + dt (S(t) + S(t + dt)) / 2,
solved by unpreconditioned GMRES(restart) with modified Gram-Schmidt Arnoldi
and Givens rotations, x_0 = u, stopping at ||b - M x|| <= tol ||b||.

Pins (tests/test_oracle_cn.py): GMRES against a direct sparse solve; one CN
step against the dense (I - dt/2 A)^{-1} (I + dt/2 A) formula; second order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class GmresStats:
    iters: int = 0
    matvecs: int = 0
    restarts: int = 0
    relres: float = 0.0
    converged: bool = True


def gmres(apply_M, b, x0, tol=1e-10, restart=50, max_iters=5000, force_iters=None):
    """Restarted GMRES with MGS-Arnoldi and Givens rotations.

    ``force_iters``: run exactly that many Arnoldi steps in one cycle
    (force_iters <= restart) and return, with no convergence test.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    st = GmresStats()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), st
    m_cap = restart if force_iters is None else force_iters
    while True:
        r = b - apply_M(x)
        st.matvecs += 1
        beta = np.linalg.norm(r)
        st.relres = beta / bnorm
        if force_iters is None and (st.relres <= tol or st.iters >= max_iters):
            st.converged = st.relres <= tol
            return x, st
        V = np.zeros((m_cap + 1, len(b)))
        H = np.zeros((m_cap + 1, m_cap))
        cs = np.zeros(m_cap)
        sn = np.zeros(m_cap)
        g = np.zeros(m_cap + 1)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m_cap):
            w = apply_M(V[k])
            st.matvecs += 1
            st.iters += 1
            for i in range(k + 1):
                H[i, k] = np.dot(V[i], w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                tmp = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = tmp
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / den
            sn[k] = H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k_used = k + 1
            if force_iters is None and (abs(g[k + 1]) <= tol * bnorm or st.iters >= max_iters):
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y
        st.restarts += 1
        if force_iters is not None:
            st.relres = abs(g[k_used]) / bnorm
            return x, st


def cn_step(A, u, t, dt, source_at, tol=1e-10, restart=50, force_iters=None):
    """One Crank-Nicolson step (reading in the module docstring)."""
    u = np.asarray(u, dtype=np.float64)
    Au = A @ u
    b = u + 0.5 * dt * Au + 0.5 * dt * (source_at(t) + source_at(t + dt))
    apply_M = lambda x: x - 0.5 * dt * (A @ x)
    x, st = gmres(apply_M, b, u, tol, restart, force_iters=force_iters)
    st.matvecs += 1
    return x, st
