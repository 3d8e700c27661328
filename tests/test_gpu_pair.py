"""The FP32 two-iteration kernel (temporal blocking) against the oracle and
against the one-iteration kernel.

On the phi_1 form (no augmented couplings), with nx % 4 == 0, ny >= 2 and no
varying advection, FP32 series run two Newton iterations per launch
(leja_iter2_f32_ring_k): y_{m+1} lives only in registers, and d_{m+2} y_{m+2}
is added to p by the next launch (or by a flush after the series).  Every
vector entry is formed by the same operations in the same order as on the
one-iteration kernel (selected with AD_F32_PAIR=0), so with the same
iteration count the results are identical.  The norm sums of the stopping
rule run over another lane-to-column assignment (120-column strips instead of
128), so the error estimates agree to FP32 rounding of the sums only.  Forced
counts of either parity also match the oracle to the FP32 bar.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import DEV, ad, devT, gpu_operator, need_gpu, oracle_operator, torch
from oracle import leja
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # (nx, ny, bc, kind, adv)
    (256, 64, BC_DIRICHLET0, "stream", (0.0, 0.0)),
    (132, 37, BC_PERIODIC, "random", (0.3, -0.2)),    # one full strip and a 4-column strip
    (8, 2, BC_DIRICHLET0, "random", (0.0, 0.0)),      # two rows: every row is a boundary row
    (4, 3, BC_PERIODIC, "uniform", (0.1, 0.0)),       # one lane, wrapped halo columns
    (516, 129, BC_DIRICHLET0, "circular", (0.2, 0.1)),
    (1024, 300, BC_PERIODIC, "stream", (0.0, 0.0)),   # several runs per warp
    (364, 50, BC_DIRICHLET0, "random", (0.0, 0.2)),   # 4 strips, right ghost group in lane 5
    (240, 33, BC_PERIODIC, "circular", (0.0, 0.0)),   # nx a multiple of the 120-column strip
]
FORCED = [1, 2, 3, 4, 9, 10]

# Runs one case on the FP32 path: forced phi_1 actions, an adaptive phi_1
# action and one- and two-stage steps; prints JSON stats, saves the vectors.
CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2307_12276_gb300 as ad
from workloads import small_problem
nx, ny, bc, kind, adv = {case!r}
p = small_problem(nx, ny, bc, kind, adv=tuple(adv), dt_factor=80.0, s=2, c=(1 / 3, 2 / 3))
T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(),
                              device="cuda:0").float()
D64 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda:0")
g = p.grid
op = ad.create_operator(g.nx, g.ny, g.bc, D64(p.Dxx), D64(p.Dxy), D64(p.Dyy), float(p.ax),
                        float(p.ay), ad.FP32_STORAGE)
v = T(np.random.default_rng(5).standard_normal(g.n))
stats, arrays = {{}}, {{}}
for m in {forced!r}:
    out = torch.empty_like(v)
    stats["f%d" % m] = ad.leja_phi1(op, v, out, p.dt, force_iters=m)
    arrays["f%d" % m] = out.cpu().numpy()
out = torch.empty_like(v)
stats["adaptive"] = ad.leja_phi1(op, v, out, p.dt, tol=1e-6)
arrays["adaptive"] = out.cpu().numpy()
src = ad.Source([D64(gk).float() for gk in p.source.g], list(p.source.h)) if len(p.source) else None
for s, c in ((1, (0.5,)), (2, (1 / 3, 2 / 3))):
    u = T(p.u0)
    stats["step%d" % s] = ad.expquad_step(op, u, 0.1, p.dt, s, c, src, tol=1e-6)
    arrays["step%d" % s] = u.cpu().numpy()
ad.time_series(op)
ad.leja_phi1(op, v, torch.empty_like(v), p.dt, tol=1e-6)
stats["path"] = ad.series_timing(op)["kernel"]
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
@pytest.mark.parametrize("march", ["0", "1", "2"])
def test_two_iteration_kernel_equals_one_iteration_kernel(case, march, tmp_path):
    """Every marching of the two-iteration kernel (0 plain, 1 with one row of
    lookahead in registers, 2 the same with the stencil levels in packed FP32
    pairs) forms the same values in the same order as the one-iteration
    kernel."""
    need_gpu()
    s2, a2 = _run(case, str(tmp_path / "pair"), {"AD_F32_MARCH": march})
    s1, a1 = _run(case, str(tmp_path / "single"), {"AD_F32_PAIR": "0"})
    assert s2["path"] == "graph loop of two-iteration kernels"
    assert s1["path"] == "graph loop of per-iteration kernels"
    for key in a1.files:
        assert s2[key]["iters"] == s1[key]["iters"], (key, s2[key], s1[key])
        assert s2[key]["converged"] == s1[key]["converged"]
        assert s2[key]["err_est"] == pytest.approx(s1[key]["err_est"], rel=1e-5, abs=1e-30), key
        assert np.array_equal(a2[key], a1[key]), key
    for m in FORCED:
        assert s2["f%d" % m]["iters"] == m


@pytest.mark.parametrize("case", [c for c in CASES if c[2] == BC_DIRICHLET0])
def test_tma_rows_equal_cp_async_rows(case, tmp_path):
    """The two-iteration kernel with its row records brought in by TMA
    (cp.async.bulk.tensor boxes, zero fill outside the grid; AD_F32_TMA=1)
    against the same kernel on per-lane cp.async rings: every record holds the
    same values, so vectors, counts and error estimates are identical."""
    need_gpu()
    st, at = _run(case, str(tmp_path / "tma"), {"AD_F32_TMA": "1"})
    sc, ac = _run(case, str(tmp_path / "cp"), {})
    assert st["path"] == "graph loop of two-iteration kernels, TMA rows"
    assert sc["path"] == "graph loop of two-iteration kernels"
    for key in ac.files:
        assert st[key]["iters"] == sc[key]["iters"], key
        assert st[key]["err_est"] == sc[key]["err_est"], key
        assert np.array_equal(at[key], ac[key]), key


@pytest.mark.parametrize("case", CASES[:4])
@pytest.mark.parametrize("m", FORCED)
def test_forced_counts_of_either_parity_match_oracle(case, m):
    """An even count leaves d_m y_m pending until the flush; an odd count stops
    after the first iteration of a launch."""
    need_gpu()
    nx, ny, bc, kind, adv = case
    p = small_problem(nx, ny, bc, kind, adv=adv, dt_factor=80.0)
    A, alpha = oracle_operator(p)
    op = gpu_operator(p, precision=1)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(12).standard_normal(p.grid.n)
    ref, _ = leja.leja_phi1(A, v, p.dt, alpha, force_iters=m)
    out = torch.empty(p.grid.n, dtype=torch.float32, device=DEV)
    st = ad().leja_phi1(op, devT(v, 1), out, p.dt, force_iters=m)
    assert st["iters"] == m
    got = out.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_profile_counts_iterations_not_launches():
    """ad_profile_leja_iteration reports time per iteration on both kernels."""
    need_gpu()
    p = small_problem(512, 512, BC_DIRICHLET0, "stream", dt_factor=80.0)
    op = gpu_operator(p, precision=1)
    t = [ad().profile_leja_iteration(op, 0, reps) for reps in (40, 41)]
    assert all(x > 0.0 for x in t)
    assert 0.5 < t[0] / t[1] < 2.0
