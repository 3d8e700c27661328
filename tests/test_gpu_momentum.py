"""The momentum-coupled operator (Eq. cr_full's momentum terms) on the GPU
against the oracle (oracle/momentum.py), through the C ABI.

Sizes span ragged grids, one momentum slice, both boundary conditions, with
and without advection, and a 128^2 x 16 case (262k unknowns).
"""
import numpy as np
import pytest

from gpu_util import DEV, ad, dev64, need_gpu, torch, assert_close
from oracle import integrators, leja, momentum, spectral
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC
from workloads.momentum import momentum_problem

pytestmark = pytest.mark.gpu

CASES = [  # (nx, ny, np, bc, kind, adv)
    (12, 10, 5, BC_DIRICHLET0, "circular", (0.3, -0.2)),
    (9, 7, 1, BC_PERIODIC, "random", (0.0, 0.0)),
    (16, 16, 12, BC_PERIODIC, "stream", (0.1, 0.05)),
    (7, 13, 3, BC_DIRICHLET0, "random", (0.0, 0.4)),
    (33, 20, 6, BC_DIRICHLET0, "spiral2", (0.0, 0.0)),
]


def _both(case, dt_factor=50.0):
    nx, ny, npm, bc, kind, adv = case
    mp = momentum_problem(nx, ny, npm, bc, kind, adv=adv, dt_factor=dt_factor)
    s = mp.spatial
    M = momentum.momentum_matrix(mp.mom.P, mp.mom.dpp, mp.mom.b, mp.mom.loss)
    A = momentum.assemble3d(s.grid, s.Dxx, s.Dxy, s.Dyy, s.ax, s.ay, mp.mom.beta, M)
    op = ad().create_momentum_operator(nx, ny, bc, dev64(s.Dxx), dev64(s.Dxy), dev64(s.Dyy),
                                       mp.mom.P, mp.mom.beta, mp.mom.dpp, mp.mom.b, mp.mom.loss,
                                       ax=s.ax, ay=s.ay)
    return mp, A, op


@pytest.mark.parametrize("case", CASES)
def test_apply_and_gershgorin_match_oracle(case):
    need_gpu()
    mp, A, op = _both(case)
    u = np.random.default_rng(4).standard_normal(A.shape[0])
    out = torch.empty(A.shape[0], dtype=torch.float64, device=DEV)
    ad().momentum_apply(op, dev64(u), out)
    assert_close(out.cpu().numpy(), A @ u, 1e-13)
    alpha = spectral.gershgorin(A)
    assert abs(ad().momentum_spectral_bound(op) - alpha) <= 1e-13 * abs(alpha)


@pytest.mark.parametrize("case", CASES)
def test_phi1_forced_and_adaptive_match_oracle(case):
    need_gpu()
    mp, A, op = _both(case)
    alpha = ad().momentum_spectral_bound(op)
    v = mp.S.ravel() + 0.1 * np.random.default_rng(5).standard_normal(A.shape[0])
    out = torch.empty(A.shape[0], dtype=torch.float64, device=DEV)
    ref, _ = leja.leja_phi1(A, v, mp.dt, alpha, force_iters=25)
    st = ad().momentum_leja_phi1(op, dev64(v), out, mp.dt, force_iters=25)
    assert st["iters"] == 25
    assert_close(out.cpu().numpy(), ref, 1e-12)
    ref, ost = leja.leja_phi1(A, v, mp.dt, alpha, tol=1e-10)
    st = ad().momentum_leja_phi1(op, dev64(v), out, mp.dt, tol=1e-10)
    assert st["iters"] == ost.iters and st["converged"] == 1
    assert_close(out.cpu().numpy(), ref, 1e-10)


def test_phi1_with_substeps_matches_oracle():
    need_gpu()
    mp, A, op = _both(CASES[0], dt_factor=400.0)
    alpha = ad().momentum_spectral_bound(op)
    ad().momentum_set_options(op, rho_max=20.0)
    v = mp.S.ravel()
    ref, ost = leja.leja_phi1(A, v, mp.dt, alpha, tol=1e-10, rho_max=20.0)
    out = torch.empty(A.shape[0], dtype=torch.float64, device=DEV)
    st = ad().momentum_leja_phi1(op, dev64(v), out, mp.dt, tol=1e-10)
    assert st["substeps"] == ost.substeps > 1 and st["iters"] == ost.iters
    assert_close(out.cpu().numpy(), ref, 1e-10)


@pytest.mark.parametrize("case", [CASES[0], CASES[2], (128, 128, 16, BC_DIRICHLET0, "circular",
                                                       (0.1, 0.05))])
def test_steps_match_oracle(case):
    """Three exponential midpoint steps with the time-independent source."""
    need_gpu()
    mp, A, op = _both(case, dt_factor=100.0)
    alpha = ad().momentum_spectral_bound(op)
    S = mp.S.ravel()
    u_ref = mp.u0.ravel().copy()
    u = dev64(u_ref)
    Sd = dev64(S)
    for _ in range(3):
        u_ref, ost = integrators.expquad_step(A, u_ref, 0.0, mp.dt, 1, (0.5,), lambda t: S,
                                              alpha, tol=1e-10)
        st = ad().momentum_step(op, u, mp.dt, Sd, tol=1e-10)
        assert st["iters"] == ost.iters and st["matvecs"] == ost.matvecs
    assert_close(u.cpu().numpy(), u_ref, 1e-10)


def test_invalid_arguments_raise():
    need_gpu()
    mp = momentum_problem(8, 8, 4)
    s = mp.spatial
    f = [dev64(s.Dxx), dev64(s.Dxy), dev64(s.Dyy)]
    m = mp.mom
    bad_P = m.P.copy()
    bad_P[2] = bad_P[1]
    with pytest.raises(ad().AdError):
        ad().create_momentum_operator(8, 8, s.grid.bc, *f, bad_P, m.beta, m.dpp, m.b, m.loss)
    with pytest.raises(ad().AdError):
        ad().create_momentum_operator(8, 8, s.grid.bc, *f, m.P, m.beta, -m.dpp, m.b, m.loss)
    with pytest.raises(ad().AdError):
        ad().create_momentum_operator(8, 8, s.grid.bc, *f, m.P[:1], m.beta[:0], m.dpp[:1],
                                      m.b[:1], m.loss[:0])
    op = ad().create_momentum_operator(8, 8, s.grid.bc, *f, m.P, m.beta, m.dpp, m.b, m.loss)
    u = dev64(mp.u0.ravel())
    with pytest.raises(ad().AdError):
        ad().momentum_apply(op, u, u)
    with pytest.raises(ad().AdError):
        ad().momentum_set_spectral_bound(op, 1.0)
