"""Pins of the penalised IMEX oracle: reduction to explicit Euler, first-order
convergence to the exact solution, stability far beyond the explicit limit,
and the exact implicit solve."""
import numpy as np
import scipy.linalg as sla

from oracle import operator as op
from oracle import penalised
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC


def _setup(bc=BC_DIRICHLET0, kind="circular", adv=(0.2, 0.1)):
    p = small_problem(12, 10, bc, kind, adv=adv)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax, p.ay)
    L = penalised.penalty_operator(p.grid)
    return p, A, L


def test_penalty_operator_is_the_isotropic_laplacian():
    """L is symmetric negative semi-definite and annihilates constants (periodic)."""
    p, A, L = _setup(bc=BC_PERIODIC)
    Ld = L.toarray()
    assert np.allclose(Ld, Ld.T, atol=1e-9)
    assert np.abs(Ld @ np.ones(p.grid.n)).max() <= 1e-9 * np.abs(Ld).max()
    assert np.linalg.eigvalsh(Ld).max() <= 1e-8 * np.abs(Ld).max()
    # interior row: the 5-point stencil 1/dx^2 (1, -2, 1) + 1/dy^2 (1, -2, 1)
    i, j = 5, 4
    row = Ld[j * p.grid.nx + i]
    assert np.isclose(row[j * p.grid.nx + i], -2 / p.grid.dx ** 2 - 2 / p.grid.dy ** 2)
    assert np.isclose(row[j * p.grid.nx + i + 1], 1 / p.grid.dx ** 2)
    assert np.isclose(row[(j + 1) * p.grid.nx + i], 1 / p.grid.dy ** 2)
    assert np.count_nonzero(np.abs(row) > 1e-12) == 5


def test_beta_zero_is_explicit_euler():
    p, A, L = _setup()
    S = lambda t: p.source_at(t).ravel()
    u = p.u0.ravel()
    dt = 0.3 * p.cfl
    got = penalised.imex_step(A, L, u, 0.2, dt, S, 0.0)
    assert np.allclose(got, u + dt * (A @ u + S(0.2)), rtol=1e-13, atol=1e-15)


def test_first_order_convergence_to_exact_solution():
    """Source-free: u(T) = exp(T A) u0; halving dt halves the error."""
    p, A, L = _setup()
    beta = penalised.default_beta(p.Dxx, p.Dxy, p.Dyy)
    u0 = p.u0.ravel()
    T = 40 * p.cfl
    exact = sla.expm(T * A.toarray()) @ u0
    zero = lambda t: np.zeros(p.grid.n)
    errs = []
    for n in (20, 40, 80):
        u = u0.copy()
        for k in range(n):
            u = penalised.imex_step(A, L, u, k * T / n, T / n, zero, beta)
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 0.85) & (rates < 1.3)), (errs, rates)


def test_stable_far_beyond_the_explicit_limit():
    """Symmetric diffusion (a = 0): the penalised step at 500 dt_CFL does not
    grow the solution; explicit Euler at the same step explodes."""
    p, A, L = _setup(adv=(0.0, 0.0))
    beta = penalised.default_beta(p.Dxx, p.Dxy, p.Dyy)
    zero = lambda t: np.zeros(p.grid.n)
    dt = 500 * p.cfl
    u = p.u0.ravel().copy()
    n0 = np.linalg.norm(u)
    for k in range(20):
        u = penalised.imex_step(A, L, u, 0.0, dt, zero, beta)
    assert np.linalg.norm(u) <= n0
    v = p.u0.ravel().copy()
    for k in range(20):
        v = v + dt * (A @ v)
    assert np.linalg.norm(v) > 1e6 * n0


def test_implicit_system_is_solved_exactly():
    p, A, L = _setup()
    beta = 2.0
    S = lambda t: p.source_at(t).ravel()
    u = p.u0.ravel()
    dt = 50 * p.cfl
    up = penalised.imex_step(A, L, u, 0.0, dt, S, beta)
    M = np.eye(p.grid.n) - dt * beta * L.toarray()
    assert np.allclose(M @ (up - u), dt * (A @ u + S(0.0)), rtol=1e-10, atol=1e-12)
