"""Pins of the oracle's Leja machinery (Section 2).

* Leja points: closed-form first points and the greedy-maximum property;
* divided differences: interpolation property, exactness on polynomials and
  agreement with 60-digit arithmetic;
* scalar phi_1: the 1x1 operator reproduces phi_1(z) = (e^z - 1)/z (recursion
  of Section 2 from phi_0 = exp);
* dense matrices: phi_1(dt A) v against exp([[dt A, v], [0, 0]]) (block
  identity) and against an eigendecomposition with scalar phi_l;
* augmented exponential: top block = dt phi_1 w1 + dt^2 phi_2 w2.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import leja
from oracle import operator as op
from oracle import spectral
from workloads import Grid, small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC


def test_first_leja_points_closed_form():
    x = leja.leja_points(8)
    assert x[0] == 2.0 and x[1] == -2.0 and abs(x[2]) < 1e-15
    # after {2, -2, 0}: maximise |xi (xi^2 - 4)| -> 4 - 3 xi^2 = 0, tie to +
    assert abs(x[3] - 2 / math.sqrt(3)) < 1e-15
    # after {2, -2, 0, 2/sqrt3}: stationary points of xi(xi^2-4)(xi-2/sqrt3)
    s = 2 / math.sqrt(3)
    poly = np.polyder(np.poly1d([1, -s, -4, 4 * s, 0]))
    roots = poly.r.real
    cand = roots[(roots > -2) & (roots < 0)]
    val = lambda t: abs(t * (t * t - 4) * (t - s))
    assert abs(x[4] - max(cand, key=val)) < 1e-13


def test_leja_greedy_maximum_on_dense_grid():
    x = leja.leja_points(80)
    grid = np.linspace(-2, 2, 400001)
    logp = np.zeros_like(grid)
    for k in range(1, 80):
        logp += np.log(np.abs(grid - x[k - 1]) + 1e-300)
        own = np.sum(np.log(np.abs(x[k] - x[:k])))
        assert own >= logp.max() - 1e-9
        assert np.min(np.abs(x[k] - x[:k])) > 0


def test_divided_differences_interpolate_and_polynomial_exact():
    x = leja.leja_points(25)
    f = np.exp(0.7 * x) * np.cos(x)
    d = leja.divided_differences(x, f)
    for t in range(25):                  # Newton form at node t reproduces f
        val, w = 0.0, 1.0
        for m in range(t + 1):
            val += d[m] * w
            w *= x[t] - x[m]
        assert abs(val - f[t]) < 1e-12
    cubic = 3 * x ** 3 - x + 0.5
    dc = leja.divided_differences(x, cubic)
    assert abs(dc[3] - 3.0) < 1e-12 and np.max(np.abs(dc[4:])) < 1e-11


@pytest.mark.parametrize("rho", [5.0, 60.0, 250.0])
def test_divided_differences_vs_high_precision(rho):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    n = 160
    x = leja.leja_points(n)
    d = leja.divided_differences(x, np.exp(rho * (x - 2)))
    X = [mpmath.mpf(v) for v in x]
    D = [mpmath.exp(rho * (v - 2)) for v in X]
    for j in range(1, n):
        for i in range(n - 1, j - 1, -1):
            D[i] = (D[i] - D[i - 1]) / (X[i] - X[i - j])
    assert max(abs(float(D[i]) - d[i]) for i in range(n)) < 1e-14


@pytest.mark.parametrize("alpha", [-1.0, -50.0, -4000.0])
@pytest.mark.parametrize("dt", [1e-3, 0.05, 0.5])
def test_scalar_phi1(alpha, dt):
    tol = 1e-12
    for frac in (0.0, 0.1, 0.5, 0.93, 1.0):
        z = alpha * frac
        A = np.array([[z]])
        out, st = leja.leja_phi1(A, np.array([1.0]), dt, alpha, tol=tol, rho_max=1e9)
        exact = float(leja.phi1_scalar(z * dt))
        assert st.converged
        assert abs(out[0] - exact) <= 20 * tol * abs(exact) + 1e-15, (z, dt, out[0], exact)


def test_scalar_phi1_error_decreases_with_terms():
    alpha, dt, z = -400.0, 0.2, -250.0
    exact = float(leja.phi1_scalar(z * dt))
    errs = [abs(leja.leja_phi1(np.array([[z]]), np.array([1.0]), dt, alpha,
                               force_iters=m, rho_max=1e9)[0][0] - exact) for m in (5, 20, 40, 80)]
    assert errs[-1] < 1e-12 and errs[0] > errs[-1]


def _dense_phi1(A, v, dt):
    n = A.shape[0]
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = dt * A
    M[:n, n] = v
    return sla.expm(M)[:n, n]          # exp([[M, v], [0, 0]]) = [[e^M, phi_1(M) v], [0, 1]]


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_DIRICHLET0])
@pytest.mark.parametrize("kind,adv", [("random", (0.0, 0.0)), ("circular", (0.4, 0.2)),
                                      ("spiral2", (1.0, 1.0))])
def test_dense_phi1(bc, kind, adv):
    p = small_problem(12, 10, bc, kind, adv=adv, adv_field=True, dt_factor=80)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    alpha = spectral.gershgorin(A)
    v = np.random.default_rng(2).standard_normal(p.grid.n)
    tol = 1e-10
    out, st = leja.leja_phi1(A, v, p.dt, alpha, tol=tol)
    ref = _dense_phi1(A.toarray(), v, p.dt)
    assert st.converged
    assert np.linalg.norm(out - ref) <= 10 * tol * np.linalg.norm(ref)


def test_dense_phi1_with_substeps():
    p = small_problem(12, 12, BC_PERIODIC, "random", dt_factor=4000)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy)
    alpha = spectral.gershgorin(A)
    v = np.random.default_rng(4).standard_normal(p.grid.n)
    out, st = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10, rho_max=50.0)
    assert st.substeps > 1
    ref = _dense_phi1(A.toarray(), v, p.dt)
    assert np.linalg.norm(out - ref) <= 1e-9 * np.linalg.norm(ref)


def test_augmented_exponential_vs_eigen_phi_functions():
    # symmetric A (a = 0, D_xy = 0): phi_l(dt A) = V phi_l(dt Lambda) V^T with
    # scalar phi_l from the recursion of Section 2.
    g = Grid(9, 8, BC_DIRICHLET0)
    rng = np.random.default_rng(8)
    A = op.assemble(g, rng.uniform(0.5, 1.0, (8, 9)), 0.0, rng.uniform(0.2, 0.6, (8, 9)))
    lam, V = np.linalg.eigh(A.toarray())
    dt = 0.02
    w1 = rng.standard_normal(g.n)
    w2 = rng.standard_normal(g.n)
    phi = lambda l: V @ np.diag([leja.phi_l_scalar(dt * t, l) for t in lam]) @ V.T
    ref = dt * phi(1) @ w1 + dt * dt * phi(2) @ w2
    alpha = spectral.gershgorin(A)
    for rho_max in (1e9, 3.0):
        top, eta, st = leja.leja_exp_augmented(A, np.zeros(g.n), np.array([0.0, 1.0]), w1, w2,
                                               dt, alpha, tol=1e-12, rho_max=rho_max)
        assert np.linalg.norm(top - ref) <= 1e-10 * np.linalg.norm(ref)
        assert abs(eta[0] - dt) < 1e-10 and abs(eta[1] - 1.0) < 1e-12


# --- adaptive substep control (a reading: the paper fixes no control) ---------------------

def _model_attempt(model, budget):
    calls = []

    def attempt(h):
        it = model(h)
        calls.append(h)
        return it <= budget, it
    return attempt, calls


def test_adaptive_rule_hand_computed_sequences():
    # iterations 100 h^2, budget 40, one initial substep: h = 1 needs 100 (rejected), h = 1/2
    # needs 25 (accepted; no growth right after a rejection), then the remainder 1/2
    attempt, calls = _model_attempt(lambda h: round(100 * h * h), 40)
    sizes, rejected, ok, flags = leja.adaptive_substeps(1.0, 1, 40, attempt)
    assert (sizes, rejected, ok, calls) == ([0.5, 0.5], 1, True, [1.0, 0.5, 0.5])
    assert flags == [False, True, True]
    # iterations 60 h, budget 40, eight initial substeps: 1/8 needs 8 (4*8 <= 40: double),
    # 1/4 needs 15 (keep), ... and the last substep is the remainder 1/8
    attempt, calls = _model_attempt(lambda h: round(60 * h), 40)
    sizes, rejected, ok, _ = leja.adaptive_substeps(1.0, 8, 40, attempt)
    assert (sizes, rejected, ok) == ([0.125, 0.25, 0.25, 0.25, 0.125], 0, True)
    # a series that never converges: give up after MAX_REJECTS + 1 attempts
    attempt, calls = _model_attempt(lambda h: 1000, 40)
    sizes, rejected, ok, _ = leja.adaptive_substeps(1.0, 1, 40, attempt)
    assert (sizes, ok) == ([], False) and rejected == leja.MAX_REJECTS + 1
    assert calls[-1] == 2.0 ** -leja.MAX_REJECTS


def test_adaptive_phi1_rejects_and_matches_dense():
    p = small_problem(12, 12, BC_PERIODIC, "random", dt_factor=4000)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy)
    alpha = spectral.gershgorin(A)
    v = np.random.default_rng(4).standard_normal(p.grid.n)
    out, st = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10, rho_max=1e9, max_iters=40,
                             adaptive=True)
    assert st.converged and st.rejected >= 3 and st.substeps == len(st.sizes) > 8
    assert abs(sum(st.sizes) - p.dt) <= 1e-13 * p.dt
    ref = _dense_phi1(A.toarray(), v, p.dt)
    assert np.linalg.norm(out - ref) <= 1e-8 * np.linalg.norm(ref)
    # the fixed rule with one substep cannot converge in 40 iterations
    _, st_fixed = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10, rho_max=1e9, max_iters=40)
    assert not st_fixed.converged


def test_adaptive_augmented_matches_eigen_phi_functions():
    g = Grid(9, 8, BC_DIRICHLET0)
    rng = np.random.default_rng(8)
    A = op.assemble(g, rng.uniform(0.5, 1.0, (8, 9)), 0.0, rng.uniform(0.2, 0.6, (8, 9)))
    lam, V = np.linalg.eigh(A.toarray())
    dt = 0.02
    w1 = rng.standard_normal(g.n)
    w2 = rng.standard_normal(g.n)
    phi = lambda l: V @ np.diag([leja.phi_l_scalar(dt * t, l) for t in lam]) @ V.T
    ref = dt * phi(1) @ w1 + dt * dt * phi(2) @ w2
    alpha = spectral.gershgorin(A)
    top, eta, st = leja.leja_exp_augmented(A, np.zeros(g.n), np.array([0.0, 1.0]), w1, w2, dt,
                                           alpha, tol=1e-12, rho_max=1e9, max_iters=8,
                                           adaptive=True)
    assert st.converged and st.rejected >= 1 and st.substeps > 1
    assert np.linalg.norm(top - ref) <= 1e-9 * np.linalg.norm(ref)
    assert abs(eta[0] - dt) < 1e-10 and abs(eta[1] - 1.0) < 1e-12


def test_adaptive_with_ample_budget_is_the_fixed_step():
    p = small_problem(12, 10, BC_DIRICHLET0, "circular", dt_factor=80)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy)
    alpha = spectral.gershgorin(A)
    v = np.random.default_rng(6).standard_normal(p.grid.n)
    fixed, st_f = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10)
    adapt, st_a = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10, adaptive=True)
    assert st_f.substeps == 1 and st_a.rejected == 0 and st_a.substeps == 1
    assert np.array_equal(fixed, adapt) and st_a.iters == st_f.iters


def test_non_finite_norms_end_the_series_unconverged():
    """A NaN input stops the series at its first term; a bound far too small
    (0.02 x Gershgorin: most of the spectrum lies far outside the Leja
    interval) makes the terms grow until the norms overflow, and the series
    must then report failure, not pass inf <= inf as converged.  With the
    true bound the same series converges."""
    p = small_problem(12, 10, BC_DIRICHLET0, "random", dt_factor=100)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    alpha = spectral.gershgorin(A)
    v = np.random.default_rng(4).standard_normal(p.grid.n)
    _, st = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-8)
    assert st.converged
    with np.errstate(over="ignore", invalid="ignore"):
        out, st = leja.leja_phi1(A, v, p.dt, 0.02 * alpha, tol=1e-8)
    assert not st.converged and st.iters < leja.MAX_ITERS
    assert np.max(np.abs(out)) > 1e100          # the terms diverged until a norm overflowed
    w = v.copy()
    w[5] = np.nan
    _, st = leja.leja_phi1(A, w, p.dt, alpha, tol=1e-8)
    assert not st.converged and st.iters == 1
