"""FP32 vectors that are only 4-byte aligned.

The one-pass series start of the FP32 step (single operator and batch)
reads the caller's state and source fields with 16-byte copies.  A caller
vector that starts at an odd float offset must take the scalar apply path
instead, and give the oracle's result."""
import numpy as np
import pytest

from gpu_util import DEV, ad, assert_close, devT, gpu_operator, need_gpu, oracle_operator, torch
from oracle import integrators
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0

pytestmark = pytest.mark.gpu


def _offset(a):
    """A float32 device copy of a whose first element sits 4 bytes past a
    16-byte boundary."""
    flat = np.ascontiguousarray(a, dtype=np.float64).ravel()
    buf = torch.zeros(flat.size + 4, dtype=torch.float32, device=DEV)
    v = buf[1:1 + flat.size]
    v.copy_(torch.as_tensor(flat, device=DEV).float())
    assert v.data_ptr() % 16 == 4 and v.is_contiguous()
    return v


@pytest.mark.parametrize("src_offset", [False, True])
def test_fp32_step_with_unaligned_state(src_offset):
    need_gpu()
    p = small_problem(64, 48, BC_DIRICHLET0, "circular", dt_factor=60)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, precision=1)
    ad().set_spectral_bound(op, alpha)
    u = _offset(p.u0)
    g0 = p.source.g[0]
    src = ad().Source([_offset(g0) if src_offset else devT(g0, 1)], None)
    st = ad().expquad_step(op, u, 0.0, p.dt, 1, (0.5,), src, force_iters=12)
    ref, ost = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,),
                                        lambda t: g0.ravel(), alpha, force_iters=12)
    assert st["matvecs"] == ost.matvecs
    assert_close(u.double().cpu().numpy(), ref, 1e-5)


def test_batch_with_one_unaligned_slice():
    need_gpu()
    probs = [small_problem(n, m, BC_DIRICHLET0, "circular", dt_factor=60) for n, m in
             ((64, 40), (48, 48), (96, 32))]
    ops, us, srcs, alphas, As = [], [], [], [], []
    for k, p in enumerate(probs):
        A, alpha = oracle_operator(p)
        op = gpu_operator(p, precision=1)
        ad().set_spectral_bound(op, alpha)
        ops.append(op)
        As.append(A)
        alphas.append(alpha)
        us.append(_offset(p.u0) if k == 1 else devT(p.u0, 1))
        srcs.append(ad().Source([devT(p.source.g[0], 1)], None))
    dt = min(p.dt for p in probs)
    batch = ad().create_batch(ops, autotune=False)
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, force_iters=9)
    for k, p in enumerate(probs):
        assert st[k]["iters"] == 9
        ref, _ = integrators.expquad_step(As[k], p.u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, p=p: p.source.g[0].ravel(), alphas[k],
                                          force_iters=9)
        assert_close(us[k].double().cpu().numpy(), ref, 1e-5, f"slice {k}")
