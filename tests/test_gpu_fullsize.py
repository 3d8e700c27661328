"""Parity at the full sizes of the 4096^2 precision-form workload and of the
128-slice batch, in the launch configurations the bench times.

Sampled cells of a forced-count step are compared with the oracle's values
of those cells, each computed on a window of radius k + 2 around the cell
(window_oracle.py; exact because a k-iteration step reaches only k + 1
cells).  Both sides use the same spectral bound, set by the test from the
fields (any negative bound defines the same Newton polynomial on both
sides).  Bars: relative L2 over the samples <= 1e-11 in FP64 and <= 1e-5 in
the FP32-storage form.
"""
import numpy as np
import pytest

from gpu_util import DEV, ad, assert_close, need_gpu, oracle_at_gpu_count, rel, torch
from oracle import integrators, spectral
from oracle import operator as oop
from window_oracle import alpha_from_fields, oracle_cell, sample_cells
from workloads import config2, config3_slices, slice_problem

pytestmark = pytest.mark.gpu


def _dev(a, prec):
    t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV)
    return t if prec == ad().FP64 else t.float()


@pytest.fixture(scope="module")
def c2():
    return config2(nx=4096)


@pytest.mark.parametrize("prec,k", [("fp32", 8), ("fp32", 7), ("fp64", 8)])
def test_config2_full_size_forced_step_sampled(c2, prec, k):
    """4096^2 stream-function workload, one midpoint step of k forced
    iterations: FP32 through the two-iteration kernel (even and odd k), FP64
    through the large-grid graph loop."""
    need_gpu()
    p = c2
    g = p.grid
    P = ad().FP32_STORAGE if prec == "fp32" else ad().FP64
    alpha = alpha_from_fields(p)
    gsrc = p.source.g[0]
    D = [torch.as_tensor(np.ascontiguousarray(f).ravel(), device=DEV)
         for f in (p.Dxx, p.Dxy, p.Dyy)]
    op = ad().create_operator(g.nx, g.ny, g.bc, D[0], D[1], D[2], 0.0, 0.0, P)
    del D
    ad().set_spectral_bound(op, alpha)
    u = _dev(p.u0, P)
    src = ad().Source([_dev(gsrc, P)], None)
    st = ad().expquad_step(op, u, 0.0, p.dt, 1, (0.5,), src, tol=1e-6, force_iters=k)
    assert st["iters"] == k and st["substeps"] == 1
    out = u.double().cpu().numpy().reshape(g.ny, g.nx)
    pts = sample_cells(g.nx, g.ny, 40, seed=11)
    got = np.array([out[j, i] for i, j in pts])
    ref = np.array([oracle_cell(p, i, j, k + 2, alpha, k, gsrc) for i, j in pts])
    bar = 1e-5 if prec == "fp32" else 1e-11
    assert_close(got, ref, bar, str((rel(got, ref), bar)))


def test_config3_full_batch_forced_step_sampled():
    """The full 128-slice batch (sides 256..2048, 178 M cells), one batched
    midpoint step of 8 forced iterations with autotuned tiles; sampled cells
    of six slices (the smallest and largest sides among them) against the
    oracle."""
    need_gpu()
    k = 8
    specs = config3_slices(128)
    sides = [side for side, _, _ in specs]
    chosen = sorted({int(np.argmin(sides)), int(np.argmax(sides)), 0, 40, 77, 127})
    probs, alphas, cfls, ops, us, srcs = {}, [], [], [], [], []
    for s, (side, dpar, dperp) in enumerate(specs):
        p = slice_problem(side, dpar, dperp, dt=1.0)
        cfls.append(p.cfl)
        g = p.grid
        D = [torch.as_tensor(np.ascontiguousarray(f).ravel(), device=DEV)
             for f in (p.Dxx, p.Dxy, p.Dyy)]
        op = ad().create_operator(g.nx, g.ny, g.bc, D[0], D[1], D[2], float(p.ax), float(p.ay),
                                  ad().FP32_STORAGE)
        del D
        alphas.append(alpha_from_fields(p))
        ad().set_spectral_bound(op, alphas[-1])
        ops.append(op)
        us.append(_dev(p.u0, ad().FP32_STORAGE))
        srcs.append(ad().Source([_dev(p.source.g[0], ad().FP32_STORAGE)], None))
        if s in chosen:
            probs[s] = p                  # the others' host fields are dropped
    # the shared step: 100 Delta t_CFL of the stiffest slice (as the bench sets it)
    dt = 100.0 * min(cfls)
    for p in probs.values():
        p.dt = dt
    batch = ad().create_batch(ops, autotune=True)
    stats = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6, force_iters=k)
    assert all(st["iters"] == k for st in stats)
    for s in chosen:
        p = probs[s]
        g = p.grid
        out = us[s].double().cpu().numpy().reshape(g.ny, g.nx)
        pts = sample_cells(g.nx, g.ny, 12, seed=100 + s)
        got = np.array([out[j, i] for i, j in pts])
        ref = np.array([oracle_cell(p, i, j, k + 2, alphas[s], k, p.source.g[0])
                        for i, j in pts])
        assert_close(got, ref, 1e-5, str((s, g.nx, rel(got, ref))))


@pytest.fixture(scope="module")
def c2_1024():
    p = config2(nx=1024, tol=1e-10)
    A = oop.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    return p, A, spectral.gershgorin(A)


def test_config2_fp64_adaptive_steps_full_vector(c2_1024):
    """The stream-function workload at 1024^2 (1 M cells: the large-grid
    graph loop of per-iteration kernels that the 4096^2 FP64 path runs), three
    adaptive exponential-midpoint steps at tol 1e-10, every cell against the
    oracle: equal iteration counts per step, 1e-11 relative L2 and
    element-wise per step (each step starts both sides from the same state)."""
    need_gpu()
    p, A, alpha = c2_1024
    g = p.grid
    D = [torch.as_tensor(np.ascontiguousarray(f).ravel(), device=DEV) for f in (p.Dxx, p.Dxy, p.Dyy)]
    op = ad().create_operator(g.nx, g.ny, g.bc, D[0], D[1], D[2], 0.0, 0.0, ad().FP64)
    ad().set_spectral_bound(op, alpha)
    src = ad().Source([_dev(p.source.g[0], ad().FP64)], None)
    S = lambda t: p.source_at(t).ravel()
    u_ref = p.u0.ravel().copy()
    for k in range(3):
        t = k * p.dt
        u = _dev(u_ref, ad().FP64)
        st = ad().expquad_step(op, u, t, p.dt, 1, (0.5,), src, tol=1e-10)
        ref, ost = integrators.expquad_step(A, u_ref, t, p.dt, 1, (0.5,), S, alpha, tol=1e-10)
        assert st["substeps"] == ost.substeps == 1

        def forced(m, u_ref=u_ref, t=t):
            r, o = integrators.expquad_step(A, u_ref, t, p.dt, 1, (0.5,), S, alpha, force_iters=m)
            return r, o.err_est
        alt = oracle_at_gpu_count(st["iters"], ost.iters, forced, 1e-10)
        assert_close(u.cpu().numpy(), ref if alt is None else alt, 1e-11, f"step {k}")
        u_ref = ref
    op.close()


def test_config2_fp32_form_against_oracle_full_vector(c2_1024):
    """The FP32-storage form of the same workload (tol 1e-6, two-iteration
    kernel) against the FP64 oracle at tol 1e-10, every cell, three steps from
    u0 on both sides: <= 1e-5 relative L2 and element-wise."""
    need_gpu()
    p, A, alpha = c2_1024
    g = p.grid
    D = [torch.as_tensor(np.ascontiguousarray(f).ravel(), device=DEV) for f in (p.Dxx, p.Dxy, p.Dyy)]
    op = ad().create_operator(g.nx, g.ny, g.bc, D[0], D[1], D[2], 0.0, 0.0, ad().FP32_STORAGE)
    ad().set_spectral_bound(op, alpha)
    src = ad().Source([_dev(p.source.g[0], ad().FP32_STORAGE)], None)
    S = lambda t: p.source_at(t).ravel()
    u = _dev(p.u0, ad().FP32_STORAGE)
    ref = p.u0.ravel().copy()
    for k in range(3):
        st = ad().expquad_step(op, u, k * p.dt, p.dt, 1, (0.5,), src, tol=1e-6)
        assert st["converged"] == 1
        ref, _ = integrators.expquad_step(A, ref, k * p.dt, p.dt, 1, (0.5,), S, alpha, tol=1e-10)
        assert_close(u.double().cpu().numpy(), ref, 1e-5, f"step {k}")
    op.close()
