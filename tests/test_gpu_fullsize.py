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

from gpu_util import DEV, ad, need_gpu, rel, torch
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
    assert rel(got, ref) <= bar, (rel(got, ref), bar)


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
        assert rel(got, ref) <= 1e-5, (s, g.nx, rel(got, ref))
