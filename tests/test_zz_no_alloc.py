"""The no-allocation variant of phi_1(dt A) v (ad_leja_phi1_noalloc).

Callers that cannot call cudaMalloc (code inside a framework that owns the
device heap, or under a no-allocation-after-start-up rule) cannot create an
operator; ad_leja_phi1_noalloc serves them from a fixed device array.  This
test calls it through the C ABI twice in a row, with different inputs, and
checks each result against the operator-based ad_leja_phi1 on the same
problem and against the FP64 CPU oracle, within the parity tolerances of the
other GPU tests (1e-12 for a forced count, 1e-11 for the adaptive stopping
rule, relative L2 and element-wise).  It also checks the call in place (v and
out the same buffer), that an oversized grid is refused with a clear error,
and that a zero operator (no negative Gershgorin bound) is refused.
The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_util import (DEV, ad, assert_close, dev64, need_gpu, oracle_at_gpu_count,
                      oracle_operator, torch)
from oracle import leja
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
        assert_close(out.cpu().numpy(), ref, 1e-12)
        # the FP64 CPU oracle with the same bound
        A, _ = oracle_operator(p)
        oref, ost = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10,
                                   force_iters=force if force >= 0 else None)
        if force >= 0:
            assert st["iters"] == force
            assert_close(out.cpu().numpy(), oref, 1e-12)
        else:
            def forced(k):
                r, o = leja.leja_phi1(A, v, p.dt, alpha, force_iters=k)
                return r, o.err_est
            alt = oracle_at_gpu_count(st["iters"], ost.iters, forced, 1e-10)
            assert_close(out.cpu().numpy(), oref if alt is None else alt, 1e-11)


def test_noalloc_in_place():
    """v and out the same device buffer (the header allows it)."""
    need_gpu()
    p = small_problem(50, 44, BC_DIRICHLET0, "random", adv=(0.2, -0.1), dt_factor=80)
    g = p.grid
    A, alpha = oracle_operator(p)
    v = np.random.default_rng(9).standard_normal(g.n)
    ref, _ = leja.leja_phi1(A, v, p.dt, alpha, force_iters=30)
    buf = dev64(v)
    st = ad().leja_phi1_noalloc(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                                buf, buf, p.dt, ax=p.ax, ay=p.ay, alpha=alpha, force_iters=30)
    torch.cuda.synchronize()
    assert st["iters"] == 30
    assert_close(buf.cpu().numpy(), ref, 1e-12)


def test_noalloc_gershgorin_default_and_limits():
    need_gpu()
    p = small_problem(40, 40, BC_DIRICHLET0, "random", adv=(0.2, 0.1), dt_factor=50)
    g = p.grid
    v = np.random.default_rng(3).standard_normal(g.n)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1_noalloc(g.nx, g.ny, g.bc, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                                dev64(v), out, p.dt, ax=p.ax, ay=p.ay, alpha=0.0, force_iters=25)
    ref, _ = _reference(p, v, p.dt, st["alpha"], 25, 1e-10)
    A, alpha = oracle_operator(p)
    assert abs(st["alpha"] - alpha) <= 1e-13 * abs(alpha)
    assert_close(out.cpu().numpy(), ref, 1e-12)
    oref, _ = leja.leja_phi1(A, v, p.dt, st["alpha"], force_iters=25)
    assert_close(out.cpu().numpy(), oref, 1e-12)
    # A == 0 (D == 0, no advection): Gershgorin gives 0, which is refused
    z = torch.zeros(g.n, dtype=torch.float64, device=DEV)
    with pytest.raises(ad().AdError) as e:
        ad().leja_phi1_noalloc(g.nx, g.ny, g.bc, z, z, z, dev64(v), out, p.dt, alpha=0.0)
    assert e.value.status == ad().AD_ERR_INVALID and "not negative" in str(e.value)
    big = small_problem(300, 300, BC_PERIODIC, "uniform")             # 90000 > 65536 cells
    x = torch.zeros(big.grid.n, dtype=torch.float64, device=DEV)
    with pytest.raises(ad().AdError) as e:
        ad().leja_phi1_noalloc(300, 300, BC_PERIODIC, dev64(big.Dxx), dev64(big.Dxy),
                               dev64(big.Dyy), x, x, big.dt)
    assert e.value.status == ad().AD_ERR_INVALID and "65536" in str(e.value)
