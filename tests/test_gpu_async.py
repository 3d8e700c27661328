"""Asynchronous steps (ad_expquad_step_async + ad_async_totals).

The asynchronous call enqueues the same kernels as ad_expquad_step and leaves
out only the synchronisations, so a run of asynchronous steps must reproduce
the synchronous steps bit for bit, with the same iteration and launch counts
in the totals.  The first case is also checked against the oracle.  Host
vectors, several substeps and adaptive control fall back to the synchronous
call and still add to the totals; a series that reaches max_iters is
reported by ad_async_totals, with its step applied as ad_expquad_step
applies it.
"""
import numpy as np
import pytest

from gpu_util import devT, gpu_operator, gpu_source, need_gpu, oracle_operator, ad, assert_close
from oracle import integrators
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu

CASES = [  # (nx, ny, bc, kind, adv, precision, s, c, dt_factor)
    (96, 80, BC_DIRICHLET0, "circular", (0.1, 0.05), 0, 2, (1 / 3, 2 / 3), 200.0),
    (64, 64, BC_PERIODIC, "uniform", (0.0, 0.0), 0, 1, (0.5,), 100.0),
    (128, 72, BC_DIRICHLET0, "stream", (0.0, 0.0), 1, 1, (0.5,), 100.0),
    (100, 36, BC_PERIODIC, "random", (0.3, -0.2), 1, 2, (1 / 3, 2 / 3), 50.0),
]


def _run(p, precision, s, c, steps, use_async, tol, u=None, setup=None):
    op = gpu_operator(p, precision)
    if setup:
        setup(op)
    src = gpu_source(p, precision)
    u = devT(p.u0, precision) if u is None else u
    stats = []
    for k in range(steps):
        if use_async:
            ad().expquad_step_async(op, u, k * p.dt, p.dt, s, c, src, tol=tol)
        else:
            stats.append(ad().expquad_step(op, u, k * p.dt, p.dt, s, c, src, tol=tol))
    tot = ad().async_totals(op) if use_async else None
    return u, stats, tot, op


@pytest.mark.parametrize("case", CASES)
def test_async_steps_equal_synchronous_steps(case):
    need_gpu()
    nx, ny, bc, kind, adv, prec, s, c, f = case
    p = small_problem(nx, ny, bc, kind, adv=adv, dt_factor=f, s=s, c=c)
    tol = 1e-10 if prec == 0 else 1e-6
    steps = 4
    ua, _, tot, _ = _run(p, prec, s, c, steps, True, tol)
    us, st, _, _ = _run(p, prec, s, c, steps, False, tol)
    assert np.array_equal(ua.cpu().numpy(), us.cpu().numpy())
    assert tot["iters"] == sum(x["iters"] for x in st)
    assert tot["matvecs"] == sum(x["matvecs"] for x in st)
    assert tot["substeps"] == steps
    # FP64 steps run whole in the tile kernel, which reports itself; an
    # unfused series adds one collect kernel
    extra = 0 if prec == 0 else steps
    assert tot["kernel_launches"] == sum(x["kernel_launches"] for x in st) + extra
    assert tot["converged"]
    assert tot["err_est"] == pytest.approx(max(x["err_est"] for x in st), rel=1e-12, abs=1e-300)


def test_async_step_matches_oracle():
    """One asynchronous two-stage FP64 step against the oracle's step."""
    need_gpu()
    p = small_problem(40, 36, BC_DIRICHLET0, "circular", adv=(0.1, 0.05), dt_factor=200.0, s=2,
                      c=(1 / 3, 2 / 3))
    A, alpha = oracle_operator(p)
    S = lambda t: p.source_at(t).ravel()
    ref, _ = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 2, (1 / 3, 2 / 3), S, alpha,
                                      tol=1e-10)
    ua, _, tot, _ = _run(p, 0, 2, (1 / 3, 2 / 3), 1, True, 1e-10,
                         setup=lambda op: ad().set_spectral_bound(op, alpha))
    assert tot["converged"] and tot["iters"] >= 2
    assert_close(ua.cpu().numpy(), ref, 1e-9)


def test_fallbacks_add_to_the_totals():
    """Host vectors, several substeps and adaptive control run synchronously
    and still report through the totals."""
    need_gpu()
    p = small_problem(64, 48, BC_DIRICHLET0, "circular", dt_factor=900.0, s=2, c=(1 / 3, 2 / 3))
    c = (1 / 3, 2 / 3)
    # several substeps (rho_max forces them)
    sub = lambda op: ad().set_options(op, rho_max=100.0)
    ua, _, tot, _ = _run(p, 0, 2, c, 2, True, 1e-10, setup=sub)
    us, st, _, _ = _run(p, 0, 2, c, 2, False, 1e-10, setup=sub)
    assert st[0]["substeps"] > 1
    assert np.array_equal(ua.cpu().numpy(), us.cpu().numpy())
    assert tot["iters"] == sum(x["iters"] for x in st)
    assert tot["substeps"] == sum(x["substeps"] for x in st)
    # host vector: staged through the library, synchronous
    uh = np.ascontiguousarray(p.u0.ravel(), dtype=np.float64)
    uh, _, toth, _ = _run(p, 0, 2, c, 2, True, 1e-10, u=uh, setup=sub)
    assert np.array_equal(uh, us.cpu().numpy())
    assert toth["iters"] == tot["iters"]
    # adaptive substep control
    ada = lambda op: ad().set_substep_control(op, 1)
    ua2, _, tot2, _ = _run(p, 0, 2, c, 2, True, 1e-10, setup=ada)
    us2, st2, _, _ = _run(p, 0, 2, c, 2, False, 1e-10, setup=ada)
    assert np.array_equal(ua2.cpu().numpy(), us2.cpu().numpy())
    assert tot2["iters"] == sum(x["iters"] for x in st2)


def test_not_converged_is_reported_by_the_totals():
    """max_iters far too small: every series stops at the cap.  The totals
    raise NotConverged; the steps were applied exactly as the synchronous
    call applies them."""
    need_gpu()
    p = small_problem(64, 64, BC_DIRICHLET0, "circular", dt_factor=200.0, s=2, c=(1 / 3, 2 / 3))
    c = (1 / 3, 2 / 3)
    cap = lambda op: ad().set_options(op, max_iters=6)
    op = gpu_operator(p, 0)
    cap(op)
    src = gpu_source(p, 0)
    ua = devT(p.u0, 0)
    for k in range(2):
        ad().expquad_step_async(op, ua, k * p.dt, p.dt, 2, c, src, tol=1e-12)
    with pytest.raises(ad().NotConverged) as e:
        ad().async_totals(op)
    assert e.value.stats["converged"] == 0
    assert e.value.stats["iters"] == 2 * 6
    assert ad().async_totals(op)["iters"] == 0          # the totals were reset
    us = devT(p.u0, 0)
    op2 = gpu_operator(p, 0)
    cap(op2)
    for k in range(2):
        with pytest.raises(ad().NotConverged):
            ad().expquad_step(op2, us, k * p.dt, p.dt, 2, c, src, tol=1e-12)
    assert np.array_equal(ua.cpu().numpy(), us.cpu().numpy())


def test_series_timing_covers_async_series():
    need_gpu()
    p = small_problem(96, 80, BC_DIRICHLET0, "circular", dt_factor=200.0, s=2, c=(1 / 3, 2 / 3))
    op = gpu_operator(p, 0)
    src = gpu_source(p, 0)
    u = devT(p.u0, 0)
    ad().time_series(op)
    for k in range(3):
        ad().expquad_step_async(op, u, k * p.dt, p.dt, 2, (1 / 3, 2 / 3), src, tol=1e-10)
    tot = ad().async_totals(op)
    t = ad().series_timing(op)
    assert t["series"] == 3
    assert t["iters"] == tot["iters"]
    assert t["ms"] > 0.0
    assert t["kernel"] == "leja_cluster_f64_k"      # 96 x 80: one thread-block cluster
    ad().time_series(op, False)
