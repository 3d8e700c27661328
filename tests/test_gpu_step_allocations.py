"""No step allocates device memory.

Once an operator is created (and, for Crank-Nicolson, its GMRES basis
reserved), every step call runs on library-owned memory: the workspace and
the host-pointer staging buffers come from ad_create_operator, the basis
from ad_reserve_gmres, and ad_penalty_beta reduces on the device with no
scratch buffer.  After one warm-up call of each kind (the first step of a
kind instantiates its CUDA graph), ten more of each must leave the device's
free memory exactly unchanged.
"""
import pytest

from gpu_util import ad, dev64, devT, gpu_operator, gpu_source, need_gpu, torch
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0

pytestmark = pytest.mark.gpu


def test_steps_allocate_nothing():
    need_gpu()
    p = small_problem(96, 80, BC_DIRICHLET0, "circular", adv=(0.1, 0.05), dt_factor=100,
                      s=2, c=(1 / 3, 2 / 3), tds=True)
    big = small_problem(600, 600, BC_DIRICHLET0, "stream", dt_factor=100)   # graph-loop path
    op = gpu_operator(p)
    opb = gpu_operator(big)
    op32 = gpu_operator(big, precision=1)
    ad().reserve_gmres(op, 30)
    src, srcb, src32 = gpu_source(p), gpu_source(big), gpu_source(big, 1)
    u, ub, u32 = dev64(p.u0), dev64(big.u0), devT(big.u0, 1)
    uh = p.u0.ravel().copy()                       # host pointer: staged by the library
    out = torch.empty_like(u)
    D = (dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy))

    def calls(k):
        t = 0.01 * k
        ad().expquad_step(op, u, t, p.dt, 2, p.c, src, tol=1e-10)
        ad().expquad_step(op, uh, t, p.dt, 1, (0.5,), src, tol=1e-10)
        ad().expquad_step_async(op, u, t, p.dt, 2, p.c, src, tol=1e-10)
        ad().async_totals(op)
        ad().leja_phi1(op, u, out, p.dt, tol=1e-10)
        ad().expquad_step(opb, ub, t, big.dt, 1, (0.5,), srcb, tol=1e-10)
        ad().expquad_step(op32, u32, t, big.dt, 1, (0.5,), src32, tol=1e-6)
        ad().cn_step(op, u, t, p.dt, src, gmres_tol=1e-10, restart=30)
        ad().penalised_step(op, u, t, p.dt, src, beta=1.0, cg_tol=1e-10)
        ad().penalty_beta(p.grid.nx, p.grid.ny, *D)
        ad().apply(op, u, out)

    calls(0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for k in range(1, 11):
        calls(k)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
    # the GMRES basis is a reservation, not a lazy allocation
    with pytest.raises(ad().AdError) as e:
        ad().cn_step(op, u, 0.0, p.dt, src, gmres_tol=1e-10, restart=40)
    assert e.value.status == ad().AD_ERR_INVALID and "ad_reserve_gmres" in str(e.value)
    for o in (op, opb, op32):
        o.close()
