"""Failure detection without faulting the GPU: bounded device waits give up
with a status the host reads; NaN inputs stop a Leja series with
NOT_CONVERGED; the context stays usable afterwards."""
import numpy as np
import pytest

from gpu_util import DEV, ad, gpu_operator, need_gpu, oracle_operator, torch
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    need_gpu()
    assert ad().check_wait_timeout(50.0) == ad().AD_ERR_TIMEOUT
    assert "gave up" in ad().last_error()
    x = torch.ones(1000, device=DEV)              # the context still works
    assert float(x.sum()) == 1000.0
    assert ad().check_wait_timeout(20.0) == ad().AD_ERR_TIMEOUT


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_input_stops_series(precision):
    need_gpu()
    p = small_problem(48, 40, BC_DIRICHLET0, "random", dt_factor=100)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, precision)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(1).standard_normal(p.grid.n)
    v[100] = np.nan
    dtype = torch.float64 if precision == 0 else torch.float32
    vd = torch.as_tensor(v, device=DEV).to(dtype)
    out = torch.empty_like(vd)
    with pytest.raises(ad().NotConverged) as e:
        ad().leja_phi1(op, vd, out, p.dt, tol=1e-8)
    assert e.value.stats["converged"] == 0 and e.value.stats["iters"] <= 2
    # the operator is still usable for a clean input
    vd = torch.as_tensor(np.nan_to_num(v), device=DEV).to(dtype)
    st = ad().leja_phi1(op, vd, out, p.dt, tol=1e-6)
    assert st["converged"] == 1


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx", [48, 600])            # persistent FP64 kernels / graph loop
def test_overflowing_series_is_not_converged(precision, nx):
    """A bound far too small (0.02 x Gershgorin) leaves most of the spectrum
    outside the Leja interval: the series' terms grow until the norms
    overflow.  Infinite norms must end the series as not converged (they
    would otherwise pass the stopping test inf <= inf)."""
    need_gpu()
    p = small_problem(nx, 40, BC_DIRICHLET0, "random", dt_factor=100)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, precision)
    ad().set_spectral_bound(op, 0.02 * alpha)
    v = np.random.default_rng(4).standard_normal(p.grid.n)
    dtype = torch.float64 if precision == 0 else torch.float32
    vd = torch.as_tensor(v, device=DEV).to(dtype)
    out = torch.empty_like(vd)
    with pytest.raises(ad().NotConverged) as e:
        ad().leja_phi1(op, vd, out, p.dt, tol=1e-8)
    assert e.value.stats["converged"] == 0
