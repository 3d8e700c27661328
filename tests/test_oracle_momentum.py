"""Pins of the momentum-coupled oracle operator (Eq. cr_full readings).

Each pin is fixed by mathematics, not by re-typing the oracle's formulas:
conservation of particles, the steady state of the momentum diffusion, the
Kronecker-sum structure of exp(tA), second-order convergence against a
symbolic derivative, the direction of the upwind loss flux and the decay of
the loss term.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import leja, momentum, spectral
from oracle import operator as op
from workloads import Grid, small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC
from workloads.momentum import momentum_inputs, momentum_problem


def _setup(bc=BC_PERIODIC, npm=5, adv=(0.3, -0.2), beta=None, **kw):
    sp_ = small_problem(6, 5, bc, "random", adv=adv)
    mom = momentum_inputs(npm, **kw)
    b = mom.beta if beta is None else beta
    M = momentum.momentum_matrix(mom.P, mom.dpp, mom.b, mom.loss)
    A = momentum.assemble3d(sp_.grid, sp_.Dxx, sp_.Dxy, sp_.Dyy, sp_.ax, sp_.ay, b, M)
    return sp_, mom, M, A


def test_particle_conservation_without_losses():
    """Periodic space, no loss: sum_k dP_k sum_i (A u)_{k,i} = 0 for every u."""
    sp_, mom, M, A = _setup(loss=0.0)
    _, dP = momentum.centres(mom.P)
    w = np.repeat(dP, sp_.grid.n)
    col = w @ A.toarray()
    assert np.abs(col).max() <= 1e-12 * np.abs(A).max()
    # with losses the weighted sums are exactly -L_k dP_k
    sp_, mom, M, A = _setup(loss=3.0)
    col = w @ A.toarray()
    assert np.allclose(col, -3.0 * w, rtol=1e-12, atol=1e-12 * np.abs(A).max())


def test_steady_state_of_momentum_diffusion():
    """d/dp(p^2 Dpp d/dp(u/p^2)) vanishes for u = p^2, with any Dpp."""
    P = np.geomspace(1.0, 300.0, 9)
    p, _ = momentum.centres(P)
    rng = np.random.default_rng(0)
    M = momentum.momentum_matrix(P, rng.uniform(0.5, 2.0, 9), np.zeros(9), np.zeros(8))
    assert np.abs(M @ p ** 2).max() <= 1e-12 * np.abs(M).max() * p.max() ** 2
    assert np.abs(M @ p).max() > 1e-3 * np.abs(M).max()     # and not for u = p


def test_kronecker_sum_structure():
    """beta = 1: A = I (x) A_xy + M (x) I, so exp(tA)(v_p (x) v_x) = (e^{tM} v_p) (x) (e^{tA_xy} v_x)."""
    sp_, mom, M, A = _setup(bc=BC_DIRICHLET0, npm=4, beta=np.ones(4))
    Axy = op.assemble(sp_.grid, sp_.Dxx, sp_.Dxy, sp_.Dyy, sp_.ax, sp_.ay).toarray()
    rng = np.random.default_rng(1)
    vp, vx = rng.standard_normal(4), rng.standard_normal(sp_.grid.n)
    t = 2e-3
    lhs = sla.expm(t * A.toarray()) @ np.kron(vp, vx)
    rhs = np.kron(sla.expm(t * M) @ vp, sla.expm(t * Axy) @ vx)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


def test_momentum_diffusion_second_order():
    """Interior cells converge at second order to the symbolic derivative."""
    sympy = pytest.importorskip("sympy")
    ps = sympy.symbols("p", positive=True)
    u_expr = ps ** 3 * sympy.exp(-ps / 20)
    dpp_expr = ps ** 2
    exact = sympy.diff(ps ** 2 * dpp_expr * sympy.diff(u_expr / ps ** 2, ps), ps)
    u_f = sympy.lambdify(ps, u_expr, "numpy")
    d_f = sympy.lambdify(ps, dpp_expr, "numpy")
    e_f = sympy.lambdify(ps, exact, "numpy")
    errs = []
    for npm in (32, 64, 128):
        P = np.geomspace(1.0, 100.0, npm + 1)
        p, _ = momentum.centres(P)
        M = momentum.momentum_matrix(P, d_f(P), np.zeros(npm + 1), np.zeros(npm))
        got = M @ u_f(p)
        inner = slice(npm // 8, npm - npm // 8)
        errs.append(np.abs(got[inner] - e_f(p[inner])).max() / np.abs(e_f(p[inner])).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


def test_upwind_loss_moves_particles_down_in_momentum():
    """b < 0 (losses): a spike in cell k feeds cell k - 1 only."""
    P = np.geomspace(1.0, 100.0, 7)
    b = -0.5 * P ** 2
    M = momentum.momentum_matrix(P, np.zeros(7), b, np.zeros(6))
    e = np.zeros(6)
    e[3] = 1.0
    r = M @ e
    assert r[2] > 0 and r[3] < 0 and r[4] == 0 and r[1] == 0
    # b > 0 (reacceleration-like drift): feeds cell k + 1 only
    M = momentum.momentum_matrix(P, np.zeros(7), -b, np.zeros(6))
    r = M @ e
    assert r[4] > 0 and r[3] < 0 and r[2] == 0


def test_loss_term_decay():
    """Only losses: each slice decays as exp(-L_k t) (the Leja phi_1 series as well)."""
    sp_ = small_problem(5, 4, BC_PERIODIC, "random")
    L = np.array([1.0, 2.5, 4.0])
    M = momentum.momentum_matrix(np.array([1.0, 2.0, 4.0, 8.0]), np.zeros(4), np.zeros(4), L)
    zero = np.zeros_like(sp_.Dxx)
    A = momentum.assemble3d(sp_.grid, zero, zero, zero, 0.0, 0.0, np.ones(3), M)
    u = np.random.default_rng(2).standard_normal(3 * sp_.grid.n)
    t = 0.7
    want = np.repeat(np.exp(-L * t), sp_.grid.n) * u
    assert np.allclose(sla.expm(t * A.toarray()) @ u, want, rtol=1e-12, atol=1e-14)
    alpha = spectral.gershgorin(A)
    out, st = leja.leja_phi1(A, u, t, alpha, tol=1e-12)
    want_phi = np.repeat(np.expm1(-L * t) / (-L * t), sp_.grid.n) * u
    assert st.converged and np.allclose(out, want_phi, rtol=1e-10)


def test_coupled_phi1_matches_dense():
    """The Leja phi_1 series on the coupled operator reproduces the dense result."""
    mp = momentum_problem(6, 5, 4, dt_factor=50.0)
    g = mp.spatial.grid
    M = momentum.momentum_matrix(mp.mom.P, mp.mom.dpp, mp.mom.b, mp.mom.loss)
    A = momentum.assemble3d(g, mp.spatial.Dxx, mp.spatial.Dxy, mp.spatial.Dyy, mp.spatial.ax,
                            mp.spatial.ay, mp.mom.beta, M)
    alpha = spectral.gershgorin(A)
    v = mp.S.ravel()
    out, st = leja.leja_phi1(A, v, mp.dt, alpha, tol=1e-11)
    N = A.shape[0]
    Z = np.zeros((N + 1, N + 1))
    Z[:N, :N] = mp.dt * A.toarray()
    Z[:N, N] = v
    ref = sla.expm(Z)[:N, N]
    assert st.converged
    assert np.linalg.norm(out - ref) <= 1e-9 * np.linalg.norm(ref)
