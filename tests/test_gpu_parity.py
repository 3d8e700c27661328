"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (FP64 path): the operator pass is 9 products summed in another
order than the CSR product, so elementwise agreement is a few ulps of
|A||u|, bounded here by 1e-13 relative L2 on white-noise inputs; Leja series
and steps run with the same alpha (injected from the oracle) and the same
iteration counts agree to <= 1e-11 relative L2 per step, the bar the method
needs.  FP32-storage path: <= 1e-5 against the FP64 oracle.
"""
import numpy as np
import pytest

from gpu_util import (DEV, ad, assert_close, dev64, devT, gpu_operator, gpu_source, need_gpu,
                      oracle_at_gpu_count, oracle_operator, torch)
from oracle import cn as ocn
from oracle import integrators, leja, spectral
from workloads import config0, config1, small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu

CASES = [  # (nx, ny, bc, kind, adv, adv_field)
    (17, 23, BC_PERIODIC, "random", (0.5, -0.3), True),
    (17, 23, BC_DIRICHLET0, "random", (0.5, -0.3), True),
    (64, 64, BC_PERIODIC, "uniform", (0.0, 0.0), False),
    (96, 40, BC_DIRICHLET0, "circular", (0.1, 0.05), False),
    (300, 257, BC_DIRICHLET0, "stream", (0.0, 0.0), False),
    (33, 31, BC_PERIODIC, "spiral2", (1.0, 2.0), False),
]
TINY = [(1, 1, BC_PERIODIC), (1, 1, BC_DIRICHLET0), (2, 3, BC_PERIODIC), (1, 7, BC_DIRICHLET0),
        (9, 1, BC_PERIODIC), (2, 2, BC_DIRICHLET0)]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("case", CASES + [c + ("random", (0.3, 0.2), True) for c in TINY])
@pytest.mark.parametrize("precision", [0, 1])
def test_apply_matches_csr(case, precision):
    nx, ny, bc, kind, adv, advf = case
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf)
    A, _ = oracle_operator(p)
    op = gpu_operator(p, precision)
    u = np.random.default_rng(nx * 7 + ny).standard_normal(p.grid.n)
    ud = devT(u, precision)
    out = torch.empty_like(ud)
    ad().apply(op, ud, out)
    ref = A @ u
    tol = 1e-13 if precision == 0 else 2e-6
    assert_close(out.cpu().numpy(), ref, tol)


@pytest.mark.parametrize("case", CASES[:4] + [c + ("random", (0.3, 0.2), True) for c in TINY])
@pytest.mark.parametrize("precision", [0, 1])
def test_gershgorin_matches_oracle(case, precision):
    nx, ny, bc, kind, adv, advf = case
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, precision)
    # magnitude of the individual weights (A itself may cancel to exactly zero)
    scale = (np.abs(p.Dxx).max() / p.grid.dx ** 2 + np.abs(p.Dyy).max() / p.grid.dy ** 2
             + np.abs(p.Dxy).max() / (p.grid.dx * p.grid.dy) + 1.0)
    if abs(alpha) <= 1e-12 * scale:
        # one periodic cell: A is the zero matrix up to rounding, so the bound is
        # zero to within rounding on either side; a non-negative bound is refused
        try:
            a = ad().spectral_bound(op, ad().BOUND_GERSHGORIN)
            assert abs(a) <= 1e-12 * scale
        except ad().AdError:
            pass
        return
    a = ad().spectral_bound(op, ad().BOUND_GERSHGORIN)
    assert abs(a - alpha) <= (1e-13 if precision == 0 else 1e-6) * abs(alpha)


@pytest.mark.parametrize("use_x0", [False, True])
def test_power_iteration_matches_oracle(use_x0):
    p = small_problem(40, 37, BC_DIRICHLET0, "circular", adv=(0.1, 0.0))
    A, _ = oracle_operator(p)
    op = gpu_operator(p)
    x0 = np.random.default_rng(3).standard_normal(p.grid.n) if use_x0 else \
        spectral.splitmix64_uniform(p.grid.n, 12345)
    a_ref, est = spectral.power_iteration(A, x0, iters=40, safety=1.1)
    a = ad().spectral_bound(op, ad().BOUND_POWER, x0=dev64(x0) if use_x0 else None, seed=12345,
                            power_iters=40, safety=1.1)
    assert abs(a - a_ref) <= 1e-11 * abs(a_ref)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("m", [1, 7, 40])
def test_leja_phi1_forced_iterations(case, m):
    nx, ny, bc, kind, adv, advf = case
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf, dt_factor=150)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(5).standard_normal(p.grid.n)
    ref, _ = leja.leja_phi1(A, v, p.dt, alpha, force_iters=m)
    out = torch.empty(p.grid.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, dev64(v), out, p.dt, force_iters=m)
    assert st["iters"] == m
    assert_close(out.cpu().numpy(), ref, 1e-12)


@pytest.mark.parametrize("case", CASES)
def test_leja_phi1_adaptive(case):
    nx, ny, bc, kind, adv, advf = case
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf, dt_factor=300)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(6).standard_normal(p.grid.n)
    ref, ost = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10)
    out = torch.empty(p.grid.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, dev64(v), out, p.dt, tol=1e-10)
    assert st["substeps"] == ost.substeps == 1

    def forced(k):
        r, s = leja.leja_phi1(A, v, p.dt, alpha, force_iters=k)
        return r, s.err_est
    alt = oracle_at_gpu_count(st["iters"], ost.iters, forced, 1e-10)
    assert_close(out.cpu().numpy(), ref if alt is None else alt, 1e-11)


def test_leja_phi1_substeps_forced():
    p = small_problem(48, 40, BC_PERIODIC, "random", adv=(0.2, 0.1), dt_factor=5000)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    ad().set_options(op, rho_max=30.0)
    v = np.random.default_rng(8).standard_normal(p.grid.n)
    ref, ost = leja.leja_phi1(A, v, p.dt, alpha, force_iters=25, rho_max=30.0)
    out = torch.empty(p.grid.n, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, dev64(v), out, p.dt, force_iters=25)
    assert st["substeps"] == ost.substeps > 1 and st["matvecs"] == ost.matvecs
    assert_close(out.cpu().numpy(), ref, 1e-12)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("s,c", [(1, (0.5,)), (2, (1 / 3, 2 / 3)),
                                 (2, (0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)))])
def test_expquad_step_forced(case, s, c):
    nx, ny, bc, kind, adv, advf = case
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf, dt_factor=120, s=s, c=c)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    u = dev64(p.u0)
    S = lambda t: p.source_at(t).ravel()
    ref, ost = integrators.expquad_step(A, p.u0.ravel(), 0.13, p.dt, s, c, S, alpha,
                                        force_iters=30)
    st = ad().expquad_step(op, u, 0.13, p.dt, s, c, gpu_source(p), force_iters=30)
    assert st["matvecs"] == ost.matvecs
    assert_close(u.cpu().numpy(), ref, 1e-12)


@pytest.mark.parametrize("s,c", [(1, (0.5,)), (2, (1 / 3, 2 / 3))])
@pytest.mark.parametrize("rho_max", [200.0, 20.0])
def test_expquad_step_adaptive(s, c, rho_max):
    p = small_problem(80, 72, BC_DIRICHLET0, "circular", adv=(0.1, 0.05), dt_factor=500,
                      s=s, c=c, tds=True)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    ad().set_options(op, rho_max=rho_max)
    u = dev64(p.u0)
    S = lambda t: p.source_at(t).ravel()
    ref, ost = integrators.expquad_step(A, p.u0.ravel(), 0.05, p.dt, s, c, S, alpha, tol=1e-10,
                                        rho_max=rho_max)
    st = ad().expquad_step(op, u, 0.05, p.dt, s, c, gpu_source(p), tol=1e-10)
    assert st["substeps"] == ost.substeps
    # several substeps: the totals must agree exactly (no per-substep rerun)
    if ost.substeps == 1:
        def forced(k):
            r, o = integrators.expquad_step(A, p.u0.ravel(), 0.05, p.dt, s, c, S, alpha,
                                            force_iters=k, rho_max=rho_max)
            return r, o.err_est
        alt = oracle_at_gpu_count(st["iters"], ost.iters, forced, 1e-10)
    else:
        assert st["iters"] == ost.iters, (st, ost)
        alt = None
    assert_close(u.cpu().numpy(), ref if alt is None else alt, 1e-11)


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_DIRICHLET0])
def test_cn_step(bc):
    p = small_problem(40, 33, bc, "random", adv=(0.4, 0.2), adv_field=True, dt_factor=30)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().reserve_gmres(op, 25)
    S = lambda t: p.source_at(t).ravel()
    # exact Krylov dimension: the same approximation on both sides
    ref, _ = ocn.cn_step(A, p.u0.ravel(), 0.2, p.dt, S, force_iters=25)
    u = dev64(p.u0)
    ad().cn_step(op, u, 0.2, p.dt, gpu_source(p), force_iters=25, restart=25)
    assert_close(u.cpu().numpy(), ref, 1e-11)
    # converged solve (restarts): both meet 1e-12, so they agree far below the step error
    ref2, ost = ocn.cn_step(A, p.u0.ravel(), 0.2, p.dt, S, tol=1e-12, restart=10)
    u2 = dev64(p.u0)
    st = ad().cn_step(op, u2, 0.2, p.dt, gpu_source(p), gmres_tol=1e-12, restart=10)
    assert st["converged"] == 1 and st["iters"] > 10 and ost.iters > 10
    assert_close(u2.cpu().numpy(), ref2, 1e-10)


FP32_CASES = CASES + [
    (300, 70, BC_PERIODIC, "random", (0.4, -0.2), True),      # ragged tiles, advection field
    (513, 33, BC_DIRICHLET0, "circular", (0.2, 0.1), False),  # 3 column tiles, 2 row tiles
    (1, 40, BC_DIRICHLET0, "random", (0.0, 0.3), False),      # one column
    (257, 1, BC_PERIODIC, "random", (0.1, 0.0), False),       # one row, halo at a tile seam
]


@pytest.mark.parametrize("case", FP32_CASES)
@pytest.mark.parametrize("s", [1, 2])
def test_fp32_forced_step_matches_oracle(case, s):
    """FP32 storage and stencil arithmetic: same iteration count as the oracle,
    agreement to the FP32 bar (1e-5 relative L2)."""
    nx, ny, bc, kind, adv, advf = case
    c = (0.5,) if s == 1 else (1 / 3, 2 / 3)
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf, dt_factor=60, s=s, c=c)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, precision=1)
    ad().set_spectral_bound(op, alpha)
    S = lambda t: p.source_at(t).ravel()
    ref, ost = integrators.expquad_step(A, p.u0.ravel(), 0.1, p.dt, s, c, S, alpha, force_iters=20)
    u = devT(p.u0, 1)
    st = ad().expquad_step(op, u, 0.1, p.dt, s, c, gpu_source(p, 1), force_iters=20)
    assert st["matvecs"] == ost.matvecs
    assert_close(u.cpu().numpy(), ref, 1e-5)


@pytest.mark.parametrize("case", FP32_CASES[:6])
def test_fp32_phi1_forced_matches_oracle(case):
    nx, ny, bc, kind, adv, advf = case
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf, dt_factor=150)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, precision=1)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(11).standard_normal(p.grid.n)
    ref, _ = leja.leja_phi1(A, v, p.dt, alpha, force_iters=30)
    out = torch.empty(p.grid.n, dtype=torch.float32, device=DEV)
    ad().leja_phi1(op, devT(v, 1), out, p.dt, force_iters=30)
    assert_close(out.cpu().numpy(), ref, 1e-5)


def test_fp32_storage_step_against_fp64_oracle():
    p = small_problem(200, 180, BC_DIRICHLET0, "stream", dt_factor=100)
    A, alpha = oracle_operator(p)
    S = lambda t: p.source_at(t).ravel()
    ref, _ = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,), S, alpha, tol=1e-10)
    op = gpu_operator(p, precision=1)
    ad().set_spectral_bound(op, alpha)
    u = devT(p.u0, 1)
    st = ad().expquad_step(op, u, 0.0, p.dt, 1, (0.5,), gpu_source(p, 1), tol=1e-6)
    assert st["converged"] == 1
    assert_close(u.cpu().numpy(), ref, 1e-5)


# ------------------------------------------------------------------ edge cases
def test_zero_input_and_zero_terms():
    p = small_problem(20, 20, BC_PERIODIC, "random")
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    out = torch.full((p.grid.n,), 7.0, dtype=torch.float64, device=DEV)
    st = ad().leja_phi1(op, torch.zeros(p.grid.n, dtype=torch.float64, device=DEV), out, p.dt)
    assert st["converged"] == 1 and torch.count_nonzero(out).item() == 0
    v = np.random.default_rng(1).standard_normal(p.grid.n)
    d0 = leja.divided_differences(leja.leja_points(3), leja.phi1_scalar(
        (alpha / 2 - alpha / 4 * leja.leja_points(3)) * p.dt))[0]
    ad().leja_phi1(op, dev64(v), out, p.dt, force_iters=0)
    assert_close(out.cpu().numpy(), d0 * v, 1e-15)


def test_host_pointers_and_aliasing():
    p = small_problem(30, 26, BC_DIRICHLET0, "random", adv=(0.2, 0.1))
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(2).standard_normal(p.grid.n)
    ref, _ = leja.leja_phi1(A, v, p.dt, alpha, force_iters=20)
    host_out = np.zeros(p.grid.n)
    ad().leja_phi1(op, v.copy(), host_out, p.dt, force_iters=20)       # host in, host out
    assert_close(host_out, ref, 1e-12)
    vd = dev64(v)
    ad().leja_phi1(op, vd, vd, p.dt, force_iters=20)                   # v and out alias
    assert_close(vd.cpu().numpy(), ref, 1e-12)
    uh = p.u0.ravel().copy()                                           # host step
    ad().expquad_step(op, uh, 0.0, p.dt, 1, (0.5,), None, force_iters=10)
    refu, _ = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,),
                                       lambda t: 0 * uh, alpha, force_iters=10)
    assert_close(uh, refu, 1e-12)


def test_invalid_arguments_raise():
    p = small_problem(10, 10, BC_PERIODIC, "random")
    op = gpu_operator(p)
    x = torch.zeros(p.grid.n, dtype=torch.float64, device=DEV)
    with pytest.raises(ad().AdError):
        ad().leja_phi1(op, x, x, -1.0)
    with pytest.raises(ad().AdError):
        ad().expquad_step(op, x, 0.0, 0.1, 3, (0.5,))
    with pytest.raises(ad().AdError):
        ad().expquad_step(op, x, 0.0, 0.1, 2, (0.5, 0.5))
    with pytest.raises(ad().AdError):
        ad().set_spectral_bound(op, 1.0)
    with pytest.raises(TypeError):
        ad().apply(op, x.float(), x)
    with pytest.raises(ad().NotConverged) as e:                       # far too small alpha
        ad().set_spectral_bound(op, -1e-3)
        ad().set_options(op, max_iters=20)
        ad().leja_phi1(op, dev64(np.random.default_rng(0).standard_normal(100)), x, 50 * p.dt,
                       tol=1e-14)
    assert e.value.stats["converged"] == 0


# ------------------------------------------------------------------ full-size workloads
def test_config0_full_run_matches_oracle():
    p = config0()
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    u = dev64(p.u0)
    src = gpu_source(p)
    S = lambda t: p.source_at(t).ravel()
    ref = p.u0.ravel().copy()
    t = 0.0
    for _ in range(p.steps):
        ref, ost = integrators.expquad_step(A, ref, t, p.dt, 1, (0.5,), S, alpha, tol=1e-10)
        st = ad().expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=1e-10)
        assert st["iters"] == ost.iters
        t += p.dt
    assert_close(u.cpu().numpy(), ref, 1e-11)


@pytest.mark.parametrize("dt_factor", [50.0, 200.0, 1000.0])
def test_config1_full_size_step_matches_oracle(dt_factor):
    p = config1(dt_factor=dt_factor)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p)
    ad().set_spectral_bound(op, alpha)
    u = dev64(p.u0)
    S = lambda t: p.source_at(t).ravel()
    ref, ost = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 2, p.c, S, alpha, tol=p.tol)
    st = ad().expquad_step(op, u, 0.0, p.dt, 2, p.c, gpu_source(p), tol=p.tol)
    assert st["substeps"] == ost.substeps
    if ost.substeps == 1:
        def forced(k):
            r, o = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 2, p.c, S, alpha,
                                            force_iters=k)
            return r, o.err_est
        alt = oracle_at_gpu_count(st["iters"], ost.iters, forced, p.tol)
    else:
        assert st["iters"] == ost.iters, (st, ost)
        alt = None
    assert_close(u.cpu().numpy(), ref if alt is None else alt, 1e-11, str((st, ost)))
