"""The FP64 series of small grids in one thread-block cluster
(leja_cluster_f64_k) against the persistent tile kernel and the oracle.

Grids of up to 112^2 cells run their Newton series (the phi_1 form and the
augmented form of two-stage quadrature) -- and an exponential step of one
substep, prologue and update included -- in one cluster of up to 16 CTAs
that keeps the grid in distributed shared memory.  Every entry is formed by
the operations of the tile kernel in the same order, so with the same
iteration count the vectors are identical; the norm sums run over another
cell-to-block assignment, so the error estimates agree to rounding.
AD_F64_CLUSTER=0 selects the tile kernel.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import (DEV, ad, assert_close, dev64, gpu_operator, gpu_source, need_gpu,
                      oracle_at_gpu_count, oracle_operator, torch)
from oracle import integrators, leja
from workloads import small_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # (nx, ny, bc, kind, adv, adv_field, dt_factor)
    (64, 64, 0, "uniform", (0.0, 0.0), False, 100.0),      # the 64^2 workload's shape
    (96, 96, 1, "stream", (0.0, 0.0), False, 200.0),
    (112, 112, 0, "stream", (0.0, 0.0), False, 200.0),    # the largest cluster grid
    (100, 37, 1, "circular", (0.1, 0.05), False, 150.0),   # uneven bands (37 rows / 16)
    (17, 23, 0, "random", (0.5, -0.3), True, 50.0),        # advection field, periodic
    (4, 3, 0, "uniform", (0.1, 0.0), False, 80.0),         # three CTAs of one row
    (1, 7, 1, "random", (0.0, 0.3), False, 20.0),          # one column
]
FORCED = [1, 2, 9, 40]

# One case: forced and adaptive phi_1 actions, two midpoint and two two-stage
# steps (one launch each) and the series path; prints JSON stats, saves the
# vectors.
CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2307_12276_gb300 as ad
from workloads import small_problem
nx, ny, bc, kind, adv, advf, f = {case!r}
p = small_problem(nx, ny, bc, kind, adv=tuple(adv), adv_field=advf, dt_factor=f)
T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda:0")
g = p.grid
ax, ay = (T(p.ax_arr()), T(p.ay_arr())) if advf else (float(p.ax), float(p.ay))
op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), ax, ay, ad.FP64)
v = T(np.random.default_rng(3).standard_normal(g.n))
stats, arrays = {{}}, {{}}
ad.time_series(op)
for m in {forced!r}:
    out = torch.empty_like(v)
    stats["f%d" % m] = ad.leja_phi1(op, v, out, p.dt, force_iters=m)
    arrays["f%d" % m] = out.cpu().numpy()
out = torch.empty_like(v)
stats["adaptive"] = ad.leja_phi1(op, v, out, p.dt, tol=1e-10)
arrays["adaptive"] = out.cpu().numpy()
stats["path"] = ad.series_timing(op)["kernel"]
src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h)) if len(p.source) else None
u = T(p.u0)
for k in range(2):
    stats["step%d" % k] = ad.expquad_step(op, u, k * p.dt, p.dt, 1, (0.5,), src, tol=1e-10)
    arrays["step%d" % k] = u.cpu().numpy()
stats["step_path"] = ad.series_timing(op)["kernel"]
u = T(p.u0)
for k in range(2):
    stats["stepq%d" % k] = ad.expquad_step(op, u, k * p.dt, p.dt, 2, (1 / 3, 2 / 3), src,
                                           tol=1e-10)
    arrays["stepq%d" % k] = u.cpu().numpy()
stats["stepq_path"] = ad.series_timing(op)["kernel"]
np.savez({prefix!r}, **arrays)
print(json.dumps(stats))
"""


def _run(case, prefix, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    code = CHILD.format(root=ROOT, case=case, prefix=prefix, forced=FORCED)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(prefix + ".npz")


@pytest.mark.parametrize("case", CASES)
def test_cluster_kernel_equals_tile_kernel(case, tmp_path):
    need_gpu()
    sc, ac = _run(case, str(tmp_path / "cluster"), {})
    st, at = _run(case, str(tmp_path / "tile"), {"AD_F64_CLUSTER": "0"})
    assert sc["path"] == sc["step_path"] == sc["stepq_path"] == "leja_cluster_f64_k"
    assert st["path"] == "leja_tile_f64_k"
    for key in at.files:
        assert sc[key]["iters"] == st[key]["iters"], (key, sc[key], st[key])
        assert sc[key]["converged"] == st[key]["converged"], key
        assert sc[key]["err_est"] == pytest.approx(st[key]["err_est"], rel=1e-12, abs=1e-300), key
        assert np.array_equal(ac[key], at[key]), key
    for m in FORCED:
        assert sc["f%d" % m]["iters"] == m
    for k in range(2):   # the whole step in one launch
        assert sc["step%d" % k]["kernel_launches"] == 1
        assert sc["stepq%d" % k]["kernel_launches"] == 1


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[3]])
def test_cluster_kernel_matches_oracle(case):
    """Adaptive phi_1 at tol 1e-10 and a midpoint step against the oracle
    (1e-11, relative L2 and element-wise; equal iteration counts unless the
    stop is borderline)."""
    need_gpu()
    nx, ny, bc, kind, adv, advf, f = case
    p = small_problem(nx, ny, bc, kind, adv=adv, adv_field=advf, dt_factor=f)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, 0, adv_field=advf)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(11).standard_normal(p.grid.n)
    out = torch.empty(p.grid.n, dtype=torch.float64, device=DEV)
    ad().time_series(op)
    st = ad().leja_phi1(op, dev64(v), out, p.dt, tol=1e-10)
    assert ad().series_timing(op)["kernel"] == "leja_cluster_f64_k"
    ref, ost = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10)

    def forced(k):
        r, s = leja.leja_phi1(A, v, p.dt, alpha, force_iters=k)
        return r, s.err_est
    alt = oracle_at_gpu_count(st["iters"], ost.iters, forced, 1e-10)
    assert_close(out.cpu().numpy(), ref if alt is None else alt, 1e-11, "phi_1")

    u = dev64(p.u0)
    S = lambda t: p.source_at(t).ravel()
    st2 = ad().expquad_step(op, u, 0.0, p.dt, 1, (0.5,), gpu_source(p), tol=1e-10)
    ref2, ost2 = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,), S, alpha, 1e-10)
    assert st2["substeps"] == ost2.substeps == 1

    def forced_step(k):
        r, o = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,), S, alpha,
                                        force_iters=k)
        return r, o.err_est
    alt2 = oracle_at_gpu_count(st2["iters"], ost2.iters, forced_step, 1e-10)
    assert_close(u.cpu().numpy(), ref2 if alt2 is None else alt2, 1e-11, "midpoint step")

    # a two-stage step (the augmented series) from t = 0.1
    c = (1 / 3, 2 / 3)
    u = dev64(p.u0)
    st3 = ad().expquad_step(op, u, 0.1, p.dt, 2, c, gpu_source(p), tol=1e-10)
    assert ad().series_timing(op)["kernel"] == "leja_cluster_f64_k"
    ref3, ost3 = integrators.expquad_step(A, p.u0.ravel(), 0.1, p.dt, 2, c, S, alpha, 1e-10)
    assert st3["substeps"] == ost3.substeps == 1

    def forced_q(k):
        r, o = integrators.expquad_step(A, p.u0.ravel(), 0.1, p.dt, 2, c, S, alpha,
                                        force_iters=k)
        return r, o.err_est
    alt3 = oracle_at_gpu_count(st3["iters"], ost3.iters, forced_q, 1e-10)
    assert_close(u.cpu().numpy(), ref3 if alt3 is None else alt3, 1e-11, "two-stage step")
    op.close()
