"""Pins of the oracle's time integrators (Section 2: Eqs. exp_quad,
exp_midpoint, exp_quad_Gauss) and of Crank-Nicolson + GMRES (comparison).

* exponential midpoint is exact for a time-independent source: one step of T
  equals N steps of T/N (to the Leja tolerance);
* mass: with periodic boundaries and a divergence-free discrete flux,
  sum u+ = sum u + dt sum S(t + dt/2) to round-off (xi_0 = 2 maps to z = 0);
* a Fourier mode decays exactly as exp(lambda dt) (constant D, periodic);
* s = 2 with the paper's Gauss nodes reproduces Eq. exp_quad_Gauss term by
  term, including its printed coefficients (tests/golden/gauss_coefficients.txt);
* temporal orders 2 (midpoint, CN) and 4 (Gauss) against an independent
  high-accuracy ODE solution (scipy DOP853);
* GMRES against a direct sparse solve, one CN step against the dense formula.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import cn, integrators, leja
from oracle import operator as op
from oracle import spectral
from workloads import Grid, config0, small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _setup(p):
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    return A, spectral.gershgorin(A), (lambda t: p.source_at(t).ravel())


def test_midpoint_exact_for_time_independent_source():
    p = config0(nx=24)
    A, alpha, S = _setup(p)
    T, tol = 8 * p.dt, 1e-12
    u1, _ = integrators.expquad_step(A, p.u0.ravel(), 0.0, T, 1, (0.5,), S, alpha, tol)
    uN, _ = integrators.run(A, p.u0.ravel(), 0.0, T / 8, 8, 1, (0.5,), S, alpha, tol)
    assert np.linalg.norm(u1 - uN) <= 50 * tol * np.linalg.norm(uN)


@pytest.mark.parametrize("adv", [(0.0, 0.0), (0.8, -0.5)])
def test_mass_conservation_periodic(adv):
    p = small_problem(16, 14, BC_PERIODIC, "random", adv=adv, dt_factor=300)
    A, alpha, S = _setup(p)
    u = p.u0.ravel()
    # s = 1: exact to round-off whatever the tolerance (z = 0 is the node xi_0);
    # s = 2: the nilpotent part of the augmented matrix needs derivatives of
    # the interpolant at z = 0, so mass holds to the series tolerance there.
    for s, c, tol, bound in ((1, (0.5,), 1e-6, 1e-13), (2, (1 / 3, 2 / 3), 1e-12, 1e-10)):
        up, _ = integrators.expquad_step(A, u, 0.1, p.dt, s, c, S, alpha, tol)
        if s == 1:
            expect = u.sum() + p.dt * S(0.1 + 0.5 * p.dt).sum()
        else:  # the quadrature integrates the source with weights b_i(0)
            c1, c2 = c
            expect = u.sum() + p.dt * (c2 * S(0.1 + c1 * p.dt).sum() - c1 * S(0.1 + c2 * p.dt).sum()
                                       ) / (c2 - c1) + p.dt * 0.5 * (S(0.1 + c2 * p.dt).sum()
                                                                     - S(0.1 + c1 * p.dt).sum()) / (c2 - c1)
        assert abs(up.sum() - expect) <= bound * np.abs(up).sum()


def test_fourier_mode_decay():
    g = Grid(32, 32, BC_PERIODIC)
    Dxx, Dxy, Dyy = 0.75025, 0.43258, 0.25075
    A = op.assemble(g, Dxx, Dxy, Dyy)
    I, J = np.meshgrid(np.arange(32), np.arange(32))
    alpha = spectral.gershgorin(A)
    for kx, ky in ((1, 0), (3, 2), (16, 16), (5, 27)):
        thx, thy = 2 * np.pi * kx / 32, 2 * np.pi * ky / 32
        u0 = np.cos(thx * I + thy * J).ravel()
        lam = op.fourier_symbol(g, Dxx, Dxy, Dyy, 0.0, 0.0, thx, thy).real
        dt = 2e-3
        u1, _ = integrators.expquad_step(A, u0, 0.0, dt, 1, (0.5,), lambda t: 0 * u0, alpha, 1e-12)
        assert np.linalg.norm(u1 - math.exp(lam * dt) * u0) <= 1e-11 * np.linalg.norm(u0)


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                vals[k.strip()] = float(eval(v, {"sqrt": math.sqrt}))
    return vals


def test_gauss_step_matches_printed_formula():
    gold = _read_golden("gauss_coefficients.txt")
    c1, c2 = gold["c1"], gold["c2"]
    assert abs(c1 - 0.5 * (1 - 1 / math.sqrt(3))) < 1e-15
    g = Grid(8, 9, BC_DIRICHLET0)
    rng = np.random.default_rng(9)
    A = op.assemble(g, rng.uniform(0.5, 1, (9, 8)), 0.0, rng.uniform(0.3, 0.6, (9, 8)))
    lam, V = np.linalg.eigh(A.toarray())
    dt = 0.015
    phi = lambda l: V @ np.diag([leja.phi_l_scalar(dt * t, l) for t in lam]) @ V.T
    G1, G2 = rng.standard_normal(g.n), rng.standard_normal(g.n)
    S = lambda t: G1 * (1 + math.sin(3 * t)) + G2 * math.exp(-t)
    u = rng.standard_normal(g.n)
    t = 0.2
    S1, S2 = S(t + c1 * dt), S(t + c2 * dt)
    # Eq. exp_quad_Gauss with the printed coefficients
    ref = (u + dt * phi(1) @ (A @ u + gold["k1"] * S1 + gold["k2"] * S2)
           + dt * gold["k3"] * phi(2) @ (S2 - S1))
    got, _ = integrators.expquad_step(A, u, t, dt, 2, (c1, c2), S, spectral.gershgorin(A), 1e-13)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


def _exact_solution(A, u0, S, T):
    from scipy.integrate import solve_ivp
    Ad = A.toarray()
    sol = solve_ivp(lambda t, y: Ad @ y + S(t), (0.0, T), u0, method="DOP853",
                    rtol=1e-13, atol=1e-13)
    return sol.y[:, -1]


def test_temporal_orders():
    g = Grid(10, 10, BC_DIRICHLET0)
    X, Y = np.meshgrid(g.x0 + (np.arange(10) + .5) * g.dx, g.y0 + (np.arange(10) + .5) * g.dy)
    A = op.assemble(g, 1.0 + 0 * X, 0.2 + 0 * X, 0.6 + 0 * X, 0.3, 0.1)
    alpha = spectral.gershgorin(A)
    G = np.exp(-((X - 0.2) ** 2 + Y ** 2) / 0.1).ravel()
    S = lambda t: G * (1.0 + np.sin(2 * np.pi * t)) * 50.0
    u0 = np.exp(-(X ** 2 + (Y + 0.2) ** 2) / 0.2).ravel()
    T = 0.4
    ref = _exact_solution(A, u0, S, T)

    def err(method, n):
        u, t, dt = u0.copy(), 0.0, T / n
        for _ in range(n):
            if method == "mid":
                u, _ = integrators.expquad_step(A, u, t, dt, 1, (0.5,), S, alpha, 1e-13)
            elif method == "gauss":
                c = (0.5 * (1 - 1 / math.sqrt(3)), 0.5 * (1 + 1 / math.sqrt(3)))
                u, _ = integrators.expquad_step(A, u, t, dt, 2, c, S, alpha, 1e-13)
            else:
                u, _ = cn.cn_step(A, u, t, dt, S, tol=1e-13)
            t += dt
        return np.linalg.norm(u - ref) / np.linalg.norm(ref)

    for method, order, ns in (("mid", 2, (8, 16, 32)), ("gauss", 4, (8, 16, 32)), ("cn", 2, (8, 16, 32))):
        e = [err(method, n) for n in ns]
        slopes = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert np.all(np.abs(slopes - order) < 0.15), (method, e, slopes)


def test_gmres_matches_direct_solve():
    p = small_problem(14, 11, BC_DIRICHLET0, "random", adv=(0.5, 0.3), adv_field=True, dt_factor=30)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    M = sp.identity(p.grid.n) - 0.5 * p.dt * A
    b = np.random.default_rng(1).standard_normal(p.grid.n)
    x, st = cn.gmres(lambda v: M @ v, b, np.zeros_like(b), tol=1e-12, restart=20)
    ref = spla.spsolve(M.tocsc(), b)
    assert st.converged and st.restarts >= 1
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    # a full Krylov space solves exactly
    small = sp.identity(30) - 0.3 * sp.random(30, 30, density=0.3, random_state=2)
    b2 = np.arange(30.0)
    x2, _ = cn.gmres(lambda v: small @ v, b2, np.zeros(30), force_iters=30, restart=30)
    assert np.linalg.norm(small @ x2 - b2) <= 1e-10 * np.linalg.norm(b2)


def test_cn_step_dense_formula():
    p = small_problem(9, 7, BC_PERIODIC, "random", adv=(0.2, 0.4), dt_factor=20)
    A, alpha, S = _setup(p)
    u = p.u0.ravel()
    got, st = cn.cn_step(A, u, 0.3, p.dt, S, tol=1e-13)
    Ad = A.toarray()
    I = np.eye(p.grid.n)
    ref = np.linalg.solve(I - 0.5 * p.dt * Ad,
                          (I + 0.5 * p.dt * Ad) @ u + 0.5 * p.dt * (S(0.3) + S(0.3 + p.dt)))
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)


def test_adaptive_two_stage_step_matches_fixed_converged_step():
    """A two-stage step under adaptive substep control with a 30-iteration budget
    agrees with the same step taken by one converged series (tol 1e-12)."""
    p = small_problem(16, 14, BC_DIRICHLET0, "circular", adv=(0.3, 0.1), dt_factor=600, s=2,
                      c=(1 / 3, 2 / 3))
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    alpha = spectral.gershgorin(A)
    S = lambda t: p.source_at(t).ravel()
    ref, st_ref = integrators.expquad_step(A, p.u0.ravel(), 0.1, p.dt, 2, (1 / 3, 2 / 3), S,
                                           alpha, tol=1e-12, rho_max=1e9)
    assert st_ref.converged and st_ref.substeps == 1
    got, st = integrators.expquad_step(A, p.u0.ravel(), 0.1, p.dt, 2, (1 / 3, 2 / 3), S, alpha,
                                       tol=1e-12, rho_max=1e9, max_iters=30, adaptive=True)
    assert st.converged and st.rejected >= 1 and st.substeps > 1
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)
