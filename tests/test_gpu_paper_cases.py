"""The paper's own test problems (Section 3: rings, spirals, time-independent
and time-dependent sources) through the C ABI, checked by properties that hold
at any size: one exponential step over the whole interval reaches the
requested accuracy, the error falls with the tolerance, and the two
quadratures converge with their orders (2 for the midpoint rule, 4 for Gauss;
Eq. exp_midpoint, Eq. exp_quad_Gauss).  A small oracle comparison pins the
problem set-up itself."""
import numpy as np
import pytest

from gpu_util import ad, dev64, need_gpu, oracle_operator, rel, torch, assert_close
from oracle import integrators
from workloads.configs import paper_case

pytestmark = pytest.mark.gpu

GAUSS = (0.5 - 0.5 / 3 ** 0.5, 0.5 + 0.5 / 3 ** 0.5)


def _op(p):
    g = p.grid
    op = ad().create_operator(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy), p.ax,
                              p.ay, ad().FP64)
    src = (ad().Source([dev64(gk) for gk in p.source.g], list(p.source.h))
           if len(p.source) else None)
    return op, src


def _integrate(p, op, src, method, nsteps, tol):
    dt = p.dt / nsteps
    u = dev64(p.u0)
    for k in range(nsteps):
        if method == "gauss":
            ad().expquad_step(op, u, k * dt, dt, 2, GAUSS, src, tol=tol)
        else:
            ad().expquad_step(op, u, k * dt, dt, 1, (0.5,), src, tol=tol)
    return u.cpu().numpy()


@pytest.mark.parametrize("case", ["I", "II"])
def test_one_step_over_the_interval_meets_the_tolerance(case):
    need_gpu()
    p = paper_case(case, 48)
    op, src = _op(p)
    ref = _integrate(p, op, src, "midpoint", 1, 1e-13)
    errs = [rel(_integrate(p, op, src, "midpoint", 1, tol), ref) for tol in (1e-3, 1e-6, 1e-9)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 1e-7


@pytest.mark.parametrize("case", ["III", "IV"])
def test_quadrature_orders_on_time_dependent_sources(case):
    need_gpu()
    p = paper_case(case, 48)
    op, src = _op(p)
    ref = _integrate(p, op, src, "gauss", 64, 1e-13)
    e_mid = [rel(_integrate(p, op, src, "midpoint", n, 1e-12), ref) for n in (4, 8)]
    e_gau = [rel(_integrate(p, op, src, "gauss", n, 1e-12), ref) for n in (4, 8)]
    assert e_mid[0] / e_mid[1] > 3.0          # second order: ~4
    assert e_gau[0] / e_gau[1] > 10.0         # fourth order: ~16
    assert e_gau[1] < e_mid[1]


def test_case_II_step_matches_the_oracle():
    """One midpoint step of the spiral-2 problem with advection and the
    time-independent sources, GPU against the FP64 oracle."""
    need_gpu()
    p = paper_case("II", 24)
    A, alpha = oracle_operator(p)
    op, src = _op(p)
    ad().set_spectral_bound(op, alpha)
    dt = 50 * p.cfl
    u = dev64(p.u0)
    ad().expquad_step(op, u, 0.0, dt, 1, (0.5,), src, tol=1e-10)
    S = lambda t: p.source_at(t).ravel()
    ref, _ = integrators.expquad_step(A, p.u0.ravel(), 0.0, dt, 1, (0.5,), S, alpha, tol=1e-10)
    assert_close(u.cpu().numpy(), ref, 1e-9)
