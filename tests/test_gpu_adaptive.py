"""Adaptive substep control on the GPU against the oracle's adaptive control.

With ad_set_substep_control(op, 1) a substep whose series reaches max_iters is
rejected and retried at half the size, and cheap substeps double the next one
(oracle.leja.adaptive_substeps states the rule).  In FP64 the GPU and the
oracle take the same decisions, so the accepted and rejected counts and the
iteration totals must be equal and the results agree to the FP64 bar.
"""
import numpy as np
import pytest

from gpu_util import DEV, ad, dev64, devT, gpu_operator, gpu_source, need_gpu, oracle_operator, torch, assert_close
from oracle import integrators, leja
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu


def _adaptive_op(p, alpha, precision, max_iters, rho_max=1e9):
    op = gpu_operator(p, precision)
    ad().set_spectral_bound(op, alpha)
    ad().set_options(op, rho_max=rho_max, max_iters=max_iters)
    ad().set_substep_control(op, True)
    return op


@pytest.mark.parametrize("case", [(48, 40, BC_PERIODIC, "random", 3000.0, 40),
                                  (64, 56, BC_DIRICHLET0, "circular", 1500.0, 60)])
def test_adaptive_phi1_matches_oracle(case):
    need_gpu()
    nx, ny, bc, kind, f, budget = case
    p = small_problem(nx, ny, bc, kind, dt_factor=f)
    A, alpha = oracle_operator(p)
    v = np.random.default_rng(3).standard_normal(p.grid.n)
    ref, ost = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10, rho_max=1e9, max_iters=budget,
                              adaptive=True)
    assert ost.converged and ost.rejected >= 1 and ost.substeps > 1
    op = _adaptive_op(p, alpha, 0, budget)
    out = torch.empty(p.grid.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, dev64(v), out, p.dt, tol=1e-10)
    assert (st["substeps"], st["rejected"], st["iters"]) == (ost.substeps, ost.rejected, ost.iters)
    assert st["matvecs"] == ost.matvecs
    assert_close(out.cpu().numpy(), ref, 1e-10)


def test_adaptive_growth_matches_oracle():
    """Small initial substeps (rho_max 5) with a 100-iteration budget: cheap
    substeps double the next one, so far fewer substeps than the fixed rule."""
    need_gpu()
    p = small_problem(48, 40, BC_DIRICHLET0, "random", dt_factor=400)
    A, alpha = oracle_operator(p)
    v = np.random.default_rng(9).standard_normal(p.grid.n)
    K0 = leja.n_substeps(alpha, p.dt, 5.0)
    ref, ost = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10, rho_max=5.0, max_iters=100,
                              adaptive=True)
    assert ost.converged and ost.substeps < K0 and len(set(ost.sizes)) > 1
    op = _adaptive_op(p, alpha, 0, 100, rho_max=5.0)
    out = torch.empty(p.grid.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, dev64(v), out, p.dt, tol=1e-10)
    assert (st["substeps"], st["rejected"], st["iters"]) == (ost.substeps, ost.rejected, ost.iters)
    assert_close(out.cpu().numpy(), ref, 1e-10)


@pytest.mark.parametrize("s,c", [(1, (0.5,)), (2, (1 / 3, 2 / 3))])
def test_adaptive_step_matches_oracle(s, c):
    need_gpu()
    p = small_problem(40, 36, BC_DIRICHLET0, "circular", adv=(0.3, 0.1), dt_factor=600, s=s, c=c)
    A, alpha = oracle_operator(p)
    S = lambda t: p.source_at(t).ravel()
    ref, ost = integrators.expquad_step(A, p.u0.ravel(), 0.1, p.dt, s, c, S, alpha, tol=1e-10,
                                        rho_max=1e9, max_iters=30, adaptive=True)
    assert ost.converged and ost.rejected >= 1
    op = _adaptive_op(p, alpha, 0, 30)
    u = dev64(p.u0)
    st = ad().expquad_step(op, u, 0.1, p.dt, s, c, gpu_source(p), tol=1e-10)
    assert (st["substeps"], st["rejected"], st["iters"]) == (ost.substeps, ost.rejected, ost.iters)
    assert_close(u.cpu().numpy(), ref, 1e-10)


def test_adaptive_fp32_step_matches_oracle():
    """FP32 operator (two-iteration kernel): same rule, FP32 bar on the result."""
    need_gpu()
    p = small_problem(128, 96, BC_PERIODIC, "random", dt_factor=800)
    A, alpha = oracle_operator(p)
    S = lambda t: p.source_at(t).ravel()
    ref, ost = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,), S, alpha,
                                        tol=1e-6, rho_max=1e9, max_iters=40, adaptive=True)
    assert ost.converged and ost.rejected >= 1
    op = _adaptive_op(p, alpha, 1, 40)
    u = devT(p.u0, 1)
    st = ad().expquad_step(op, u, 0.0, p.dt, 1, (0.5,), gpu_source(p, 1), tol=1e-6)
    assert st["converged"] == 1 and st["rejected"] >= 1
    assert_close(u.cpu().numpy(), ref, 1e-5)


def test_adaptive_gives_up_and_leaves_u_unchanged():
    """A NaN input never converges: 41 rejections, AD_ERR_NOT_CONVERGED, u untouched."""
    need_gpu()
    p = small_problem(48, 40, BC_DIRICHLET0, "random", dt_factor=100)
    A, alpha = oracle_operator(p)
    op = _adaptive_op(p, alpha, 0, 100)
    u0 = p.u0.ravel().copy()
    u0[77] = np.nan
    u = dev64(u0)
    with pytest.raises(ad().NotConverged) as e:
        ad().expquad_step(op, u, 0.0, p.dt, 2, (1 / 3, 2 / 3), gpu_source(p), tol=1e-8)
    assert e.value.stats["rejected"] == leja.MAX_REJECTS + 1
    assert e.value.stats["converged"] == 0
    got = u.cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(u0))
    assert np.array_equal(got[~np.isnan(u0)], u0[~np.isnan(u0)])
    # the operator still steps a clean input
    u = dev64(p.u0)
    st = ad().expquad_step(op, u, 0.0, p.dt, 2, (1 / 3, 2 / 3), gpu_source(p), tol=1e-8)
    assert st["converged"] == 1


def test_fixed_rule_unchanged_by_default():
    """Without ad_set_substep_control the equal-substep rule applies (rejected = 0)."""
    need_gpu()
    p = small_problem(48, 40, BC_PERIODIC, "random", dt_factor=3000)
    A, alpha = oracle_operator(p)
    v = np.random.default_rng(3).standard_normal(p.grid.n)
    ref, ost = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10, rho_max=50.0)
    op = gpu_operator(p, 0)
    ad().set_spectral_bound(op, alpha)
    ad().set_options(op, rho_max=50.0)
    out = torch.empty(p.grid.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, dev64(v), out, p.dt, tol=1e-10)
    assert st["rejected"] == 0 and st["substeps"] == ost.substeps > 1
    assert_close(out.cpu().numpy(), ref, 1e-10)
