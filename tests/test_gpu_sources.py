"""FP32 midpoint steps with 0 to 3 separable source terms against the oracle.

The one-pass series start of the FP32 path (series_start_f32 for single
operators, batch_start_k for batches) takes up to two source terms through
the coupling slots of the ring run (the first through w2, the second through
w1); three or more fall back to the apply and start kernels.  Every count is
checked with forced iteration counts (both sides run the same polynomial) at
the FP32 bar, 1e-5 relative L2.  The sources are the first k terms of the
time-dependent TDS source, evaluated at t + dt/2 = 0.3 + dt/2.
"""
import numpy as np
import pytest

from gpu_util import ad, devT, gpu_operator, need_gpu, oracle_operator, assert_close
from oracle import integrators
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC, SeparableSource

pytestmark = pytest.mark.gpu

T0 = 0.3
FORCE = 6


def _problem(nx, ny, bc, terms):
    p = small_problem(nx, ny, bc, "circular", adv=(0.1, -0.05), dt_factor=50.0, tds=True)
    p.source = SeparableSource(list(p.source.g[:terms]), list(p.source.h[:terms]))
    return p


def _oracle_step(p, alpha):
    A, _ = oracle_operator(p)
    S = lambda t: p.source_at(t).ravel() if len(p.source) else np.zeros(p.grid.n)
    u, _ = integrators.expquad_step(A, p.u0.ravel(), T0, p.dt, 1, (0.5,), S, alpha, tol=1e-6,
                                    force_iters=FORCE)
    return u


def _gpu_source(p):
    if len(p.source) == 0:
        return None
    return ad().Source([devT(gk, 1) for gk in p.source.g], list(p.source.h))


@pytest.mark.parametrize("terms", [0, 1, 2, 3])
@pytest.mark.parametrize("nx,ny,bc", [(64, 48, BC_DIRICHLET0), (96, 40, BC_PERIODIC)])
def test_fp32_midpoint_source_terms(nx, ny, bc, terms):
    need_gpu()
    p = _problem(nx, ny, bc, terms)
    _, alpha = oracle_operator(p)
    ref = _oracle_step(p, alpha)
    op = gpu_operator(p, 1)
    ad().set_spectral_bound(op, alpha)
    u = devT(p.u0, 1)
    st = ad().expquad_step(op, u, T0, p.dt, 1, (0.5,), _gpu_source(p), tol=1e-6,
                           force_iters=FORCE)
    assert st["iters"] == FORCE * st["substeps"]
    assert_close(u.double().cpu().numpy(), ref, 1e-5)


@pytest.mark.parametrize("counts", [(0, 1, 2, 1), (2, 3, 0, 1)])
def test_batch_midpoint_source_terms(counts):
    """Slices with mixed source counts in one batch: up to two terms the
    one-pass start serves the batch, a slice with three sends it to the apply
    and start kernels."""
    need_gpu()
    sizes = [(64, 48), (96, 40), (128, 32), (48, 64)]
    probs = [_problem(nx, ny, BC_DIRICHLET0, k) for (nx, ny), k in zip(sizes, counts)]
    dt = min(p.dt for p in probs)
    ops, us, srcs, alphas = [], [], [], []
    for p in probs:
        p.dt = dt
        _, alpha = oracle_operator(p)
        op = gpu_operator(p, 1)
        ad().set_spectral_bound(op, alpha)
        ops.append(op)
        alphas.append(alpha)
        us.append(devT(p.u0, 1))
        srcs.append(_gpu_source(p) or ad().Source([], None))
    batch = ad().create_batch(ops, autotune=False)
    stats = ad().batch_midpoint_step(batch, us, T0, dt, srcs, tol=1e-6, force_iters=FORCE)
    assert all(s["iters"] == FORCE for s in stats)
    for p, alpha, u in zip(probs, alphas, us):
        assert_close(u.double().cpu().numpy(), _oracle_step(p, alpha), 1e-5)
