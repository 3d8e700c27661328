"""The three persistent FP64 series kernels agree bit for bit.

Small FP64 grids run a whole Newton series in one cooperative launch.  The
tile kernel (the default wherever its tiles fit in shared memory) and the row
kernel (AD_F64_KERNEL=row; the fallback) synchronise
each block with its neighbours only and apply the stopping rule two
iterations late (dropping the extra iteration); the grid-barrier kernel
(selected with AD_NO_NSYNC) decides after every iteration.  All three form
every entry of the result by the same operations, so results and iteration
counts must be identical, not merely close; the row and grid kernels also sum
the norms in the same order (identical error estimates), the tile kernel over
another cell-to-block assignment (estimates equal to rounding).  Accuracy
against the oracle is covered by the parity tests, which run the default
kernel.

Also checks the series timing counters against the step statistics.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import DEV, ad, dev64, need_gpu, oracle_operator, torch
from workloads import small_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # (nx, ny, bc, kind, adv, adv_field, dt_factor)
    (300, 257, 1, "stream", (0.0, 0.0), False, 200.0),
    (64, 64, 0, "uniform", (0.0, 0.0), False, 100.0),
    (17, 23, 0, "random", (0.5, -0.3), True, 50.0),
    (1, 7, 1, "random", (0.0, 0.3), False, 20.0),
    (513, 40, 1, "circular", (0.1, 0.05), False, 300.0),
]

# Runs one case: adaptive phi_1 action and a two-stage quadrature step, with
# the Gershgorin bound computed by the library itself.  Prints JSON stats and
# writes the two result vectors to the given .npy prefix.
CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2307_12276_gb300 as ad
from workloads import small_problem
nx, ny, bc, kind, adv, advf, f = {case!r}
p = small_problem(nx, ny, bc, kind, adv=tuple(adv), adv_field=advf, dt_factor=f, s=2,
                  c=(1 / 3, 2 / 3))
T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda:0")
g = p.grid
if advf:
    ax, ay = T(p.ax_arr()), T(p.ay_arr())
else:
    ax, ay = float(p.ax), float(p.ay)
op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), ax, ay, ad.FP64)
v = T(p.u0)
out = torch.empty_like(v)
st1 = ad.leja_phi1(op, v, out, p.dt, tol=1e-10)
u = T(p.u0)
src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h)) if len(p.source) else None
st2 = ad.expquad_step(op, u, 0.1, p.dt, 2, (1 / 3, 2 / 3), src, tol=1e-10)
np.save({prefix!r} + "_phi.npy", out.cpu().numpy())
np.save({prefix!r} + "_step.npy", u.cpu().numpy())
print(json.dumps({{"phi": st1, "step": st2}}))
"""


def _run(case, prefix, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    code = CHILD.format(root=ROOT, case=case, prefix=prefix)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    stats = json.loads(r.stdout.strip().splitlines()[-1])
    return stats, np.load(prefix + "_phi.npy"), np.load(prefix + "_step.npy")


@pytest.mark.parametrize("case", CASES)
def test_neighbour_sync_kernel_equals_grid_barrier_kernel(case, tmp_path):
    need_gpu()
    s_new, phi_new, u_new = _run(case, str(tmp_path / "nsync"), {"AD_F64_KERNEL": "row"})
    s_old, phi_old, u_old = _run(case, str(tmp_path / "grid"), {"AD_NO_NSYNC": "1"})
    for key in ("phi", "step"):
        assert s_new[key]["iters"] == s_old[key]["iters"], (key, s_new[key], s_old[key])
        assert s_new[key]["converged"] == s_old[key]["converged"]
        assert s_new[key]["err_est"] == s_old[key]["err_est"]
    assert np.array_equal(phi_new, phi_old)
    assert np.array_equal(u_new, u_old)


@pytest.mark.parametrize("case", CASES)
def test_tile_kernel_equals_grid_barrier_kernel(case, tmp_path):
    """The 2-D tile kernel forms every entry as the grid-barrier kernel does;
    its norm sums run over another cell-to-block assignment, so the error
    estimates agree to rounding."""
    need_gpu()
    s_new, phi_new, u_new = _run(case, str(tmp_path / "tile"), {"AD_F64_KERNEL": "tile"})
    s_old, phi_old, u_old = _run(case, str(tmp_path / "grid"), {"AD_NO_NSYNC": "1"})
    for key in ("phi", "step"):
        assert s_new[key]["iters"] == s_old[key]["iters"], (key, s_new[key], s_old[key])
        assert s_new[key]["converged"] == s_old[key]["converged"]
        assert s_new[key]["err_est"] == pytest.approx(s_old[key]["err_est"], rel=1e-12,
                                                      abs=1e-300)
    assert np.array_equal(phi_new, phi_old)
    assert np.array_equal(u_new, u_old)


# Two midpoint (s = 1) and two two-stage (s = 2) steps from u0; prints the
# stats of every step and writes the two final states.
STEPS_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2307_12276_gb300 as ad
from workloads import small_problem
nx, ny, bc, kind, adv, advf, f = {case!r}
out = {{}}
for s, c in ((1, (0.5,)), (2, (1 / 3, 2 / 3))):
    p = small_problem(nx, ny, bc, kind, adv=tuple(adv), adv_field=advf, dt_factor=f, s=s, c=c)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(),
                                  device="cuda:0")
    g = p.grid
    ax, ay = (T(p.ax_arr()), T(p.ay_arr())) if advf else (float(p.ax), float(p.ay))
    op = ad.create_operator(g.nx, g.ny, g.bc, T(p.Dxx), T(p.Dxy), T(p.Dyy), ax, ay, ad.FP64)
    src = ad.Source([T(gk) for gk in p.source.g], list(p.source.h)) if len(p.source) else None
    u = T(p.u0)
    st = [ad.expquad_step(op, u, k * p.dt, p.dt, s, c, src, tol=1e-10) for k in range(2)]
    np.save({prefix!r} + f"_s{{s}}.npy", u.cpu().numpy())
    out[s] = st
print(json.dumps(out))
"""


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[4]])
def test_fused_step_equals_unfused_step(case, tmp_path):
    """A whole step in one launch of the tile kernel (its prologue forms
    A u + sources as the apply kernel does, its epilogue adds P to u as the
    axpby kernel does) gives the unfused sequence's result bit for bit."""
    need_gpu()
    res = {}
    for tag, env in (("fused", {}), ("unfused", {"AD_NO_FUSE": "1"})):
        e = dict(os.environ)
        e.update(env)
        prefix = str(tmp_path / tag)
        code = STEPS_CHILD.format(root=ROOT, case=case, prefix=prefix)
        r = subprocess.run([sys.executable, "-c", code], env=e, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[tag] = (json.loads(r.stdout.strip().splitlines()[-1]),
                    {s: np.load(f"{prefix}_s{s}.npy") for s in (1, 2)})
    (sf, uf), (su, uu) = res["fused"], res["unfused"]
    for s in ("1", "2"):
        for a, b in zip(sf[s], su[s]):
            assert a["iters"] == b["iters"] and a["err_est"] == b["err_est"]
            assert a["kernel_launches"] == 1          # the whole step is one launch
            assert b["kernel_launches"] > 1
    for s in (1, 2):
        assert np.array_equal(uf[s], uu[s])


def test_series_timing_counts_every_series():
    need_gpu()
    p = small_problem(96, 80, 1, "circular", dt_factor=900.0, s=2, c=(1 / 3, 2 / 3))
    A, alpha = oracle_operator(p)
    op = ad().create_operator(p.grid.nx, p.grid.ny, p.grid.bc, dev64(p.Dxx), dev64(p.Dxy),
                              dev64(p.Dyy), 0.0, 0.0, ad().FP64)
    ad().set_spectral_bound(op, alpha)
    ad().set_options(op, rho_max=100.0)              # forces several substeps
    src = ad().Source([dev64(gk) for gk in p.source.g], list(p.source.h))
    u = dev64(p.u0)
    ad().time_series(op)
    st = ad().expquad_step(op, u, 0.0, p.dt, 2, (1 / 3, 2 / 3), src, tol=1e-10)
    t = ad().series_timing(op)
    assert st["substeps"] > 1
    assert t["series"] == st["substeps"]
    assert t["iters"] == st["iters"]
    assert t["ms"] > 0.0
    assert t["kernel"] in ("leja_cluster_f64_k", "leja_tile_f64_k", "leja_nsync_f64_k")
    ad().time_series(op, False)
    ad().expquad_step(op, u, p.dt, p.dt, 2, (1 / 3, 2 / 3), src, tol=1e-10)
    assert ad().series_timing(op) == t
    ad().time_series(op)                             # re-enabling resets the totals
    assert ad().series_timing(op) == {"ms": 0.0, "series": 0, "iters": 0, "kernel": None}


# FP64 grids across the switch points of the series path: tiles while they fit
# in shared memory, then the row or grid-barrier kernel, up to 152 x 2048 cells
# (the largest persistent grid), and the per-iteration graph loop above it.
SWITCH_SIZES = [(448, 448), (512, 512), (520, 560), (556, 558), (557, 559), (560, 560)]


def test_fp64_kernel_switch_points_match_oracle():
    """A forced two-stage step on each grid against the oracle (1e-11); the
    kernels that ran are recorded and must include the tile kernel and the
    graph loop."""
    need_gpu()
    from oracle import integrators
    seen = {}
    for nx, ny in SWITCH_SIZES:
        p = small_problem(nx, ny, 1, "circular", adv=(0.1, 0.05), dt_factor=200.0, s=2,
                          c=(1 / 3, 2 / 3))
        A, alpha = oracle_operator(p)
        S = lambda t, p=p: p.source_at(t).ravel()
        ref, _ = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 2, (1 / 3, 2 / 3), S,
                                          alpha, tol=1e-10, force_iters=12)
        op = ad().create_operator(nx, ny, 1, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy), 0.1, 0.05,
                                  ad().FP64)
        ad().set_spectral_bound(op, alpha)
        src = ad().Source([dev64(gk) for gk in p.source.g], list(p.source.h))
        u = dev64(p.u0)
        ad().time_series(op)
        st = ad().expquad_step(op, u, 0.0, p.dt, 2, (1 / 3, 2 / 3), src, tol=1e-10,
                               force_iters=12)
        kernel = ad().series_timing(op)["kernel"]
        ad().time_series(op, False)
        assert st["iters"] == 12 * st["substeps"]
        err = float(np.linalg.norm(u.cpu().numpy() - ref) / np.linalg.norm(ref))
        assert err <= 1e-11, (nx, ny, kernel, err)
        seen[(nx, ny)] = kernel
    kinds = set(seen.values())
    assert "leja_tile_f64_k" in kinds, seen
    assert seen[(560, 560)] not in ("leja_tile_f64_k", "leja_nsync_f64_k",
                                    "leja_persistent_f64_k"), seen
    print(seen)
