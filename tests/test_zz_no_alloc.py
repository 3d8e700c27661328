"""The no-allocation variant of phi_1(dt A) v (ad_leja_phi1_noalloc).

Callers that cannot call cudaMalloc (code inside a framework that owns the
device heap, or under a no-allocation-after-start-up rule) cannot create an
operator; ad_leja_phi1_noalloc serves them from a fixed device array.  This
test calls it through the C ABI twice in a row, with different inputs, and
checks each result against the operator-based ad_leja_phi1 on the same
problem, within the forced-iteration parity tolerance of the other GPU tests
(1e-12 relative L2; both run the same kernels, so the results agree far below
it).  It also checks that an oversized grid is refused with a clear error.
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_util import DEV, ad, dev64, need_gpu, rel, torch
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu


def _reference(p, v, dt, alpha, force_iters, tol):
    """Same computation through the operator-based entry point."""
    g = p.grid
    op = ad().create_operator(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                              float(p.ax), float(p.ay), ad().FP64)
    ad().set_spectral_bound(op, alpha)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, dev64(v), out, dt, tol=tol, force_iters=force_iters)
    op.close()
    return out.cpu().numpy(), st


def test_noalloc_matches_operator_entry_point_twice_in_a_row():
    need_gpu()
    calls = [
        (small_problem(64, 48, BC_DIRICHLET0, "circular", adv=(0.1, 0.05), dt_factor=120), 1, 40),
        (small_problem(96, 80, BC_PERIODIC, "random", adv=(0.3, -0.2), dt_factor=60), 2, -1),
    ]
    for p, seed, force in calls:
        g = p.grid
        v = np.random.default_rng(seed).standard_normal(g.n)
        # the spectral bound both sides use: Gershgorin of the operator-based path
        op = ad().create_operator(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                                  float(p.ax), float(p.ay), ad().FP64)
        alpha = ad().get_spectral_bound(op)
        op.close()
        ref, st_ref = _reference(p, v, p.dt, alpha, force, 1e-10)
        out = torch.full((g.n,), np.nan, dtype=torch.float64, device=DEV)
        st = ad().leja_phi1_noalloc(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                                    dev64(v), out, p.dt, ax=p.ax, ay=p.ay, alpha=alpha, tol=1e-10,
                                    force_iters=force)
        torch.cuda.synchronize()
        assert st["iters"] == st_ref["iters"]
        assert rel(out.cpu().numpy(), ref) <= 1e-12


def test_noalloc_gershgorin_default_and_limits():
    need_gpu()
    p = small_problem(40, 40, BC_DIRICHLET0, "random", adv=(0.2, 0.1), dt_factor=50)
    g = p.grid
    v = np.random.default_rng(3).standard_normal(g.n)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1_noalloc(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                                dev64(v), out, p.dt, ax=p.ax, ay=p.ay, alpha=0.0, force_iters=25)
    ref, _ = _reference(p, v, p.dt, st["alpha"], 25, 1e-10)
    assert st["alpha"] < 0 and rel(out.cpu().numpy(), ref) <= 1e-12
    big = small_problem(300, 300, BC_PERIODIC, "uniform")             # 90000 > 65536 cells
    x = torch.zeros(big.grid.n, dtype=torch.float64, device=DEV)
    with pytest.raises(ad().AdError) as e:
        ad().leja_phi1_noalloc(300, 300, BC_PERIODIC, dev64(big.Dxx), dev64(big.Dxy),
                               dev64(big.Dyy), x, x, big.dt)
    assert e.value.status == ad().AD_ERR_INVALID and "65536" in str(e.value)
