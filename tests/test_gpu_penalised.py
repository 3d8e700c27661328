"""The penalised IMEX step on the GPU (conjugate gradients on I - dt beta L)
against the oracle's exact sparse solve, through the C ABI."""
import numpy as np
import pytest

from gpu_util import ad, dev64, gpu_operator, gpu_source, need_gpu, oracle_operator, assert_close
from oracle import penalised
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu

CASES = [  # (nx, ny, bc, kind, adv, dt_factor)
    (40, 36, BC_DIRICHLET0, "circular", (0.3, 0.1), 50.0),
    (33, 17, BC_PERIODIC, "random", (0.0, 0.0), 200.0),
    (64, 64, BC_DIRICHLET0, "stream", (0.1, -0.2), 500.0),
    (1, 9, BC_PERIODIC, "random", (0.0, 0.2), 20.0),
]


@pytest.mark.parametrize("case", CASES)
def test_penalised_steps_match_oracle(case):
    need_gpu()
    nx, ny, bc, kind, adv, f = case
    p = small_problem(nx, ny, bc, kind, adv=adv, dt_factor=f)
    A, alpha = oracle_operator(p)
    L = penalised.penalty_operator(p.grid)
    beta = penalised.default_beta(p.Dxx, p.Dxy, p.Dyy)
    assert abs(ad().penalty_beta(nx, ny, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy)) - beta) \
        <= 1e-14 * beta
    op = gpu_operator(p, 0)
    S = lambda t: p.source_at(t).ravel()
    u_ref = p.u0.ravel().copy()
    u = dev64(u_ref)
    for k in range(3):
        t = k * p.dt
        u_ref = penalised.imex_step(A, L, u_ref, t, p.dt, S, beta)
        st = ad().penalised_step(op, u, t, p.dt, gpu_source(p), beta=beta, cg_tol=1e-13)
        assert st["converged"] == 1 and st["iters"] > 0
    assert_close(u.cpu().numpy(), u_ref, 1e-10)


def test_beta_zero_is_explicit_euler_and_cg_cap():
    need_gpu()
    p = small_problem(24, 20, BC_DIRICHLET0, "random", dt_factor=0.3)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, 0)
    u0 = p.u0.ravel()
    u = dev64(u0)
    st = ad().penalised_step(op, u, 0.0, p.dt, gpu_source(p), beta=0.0)
    want = u0 + p.dt * (A @ u0 + p.source_at(0.0).ravel())
    assert_close(u.cpu().numpy(), want, 1e-12 and st["iters"] <= 8)
    # a CG budget that cannot reach the tolerance: error, u unchanged
    u = dev64(u0)
    with pytest.raises(ad().NotConverged):
        ad().penalised_step(op, u, 0.0, 200 * p.dt, gpu_source(p), beta=1.0, cg_tol=1e-14,
                            max_cg=2)
    assert np.array_equal(u.cpu().numpy(), u0)
