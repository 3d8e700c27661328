"""The norms' sums of squares of the large-grid FP64 iteration, formed on the
integer and FP32 pipes (csrc/sqsum.cuh) instead of by FP64 FMAs.

They feed only the stopping rule |d| ||y|| <= tol ||p|| (Section 2): the
vectors y and p are the same FP64 values either way.  So against the same
iteration with FP64 FMA sums (AD_F64_NORMS=fp64) every vector must be equal
bit for bit with equal iteration counts, and the error estimates must agree
to the accuracy of the sums.  Scaling the input by a power of two scales
every FP64 operation exactly, and the sums split off the exponent, so the
results scale exactly and the counts and estimates do not change; the
estimate also matches the oracle's FP64 one.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import (ad, assert_close, dev64, need_gpu, oracle_at_gpu_count,
                      oracle_operator, torch)
from oracle import leja
from workloads import small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# grids above 152 x 2048 cells, where FP64 series run the per-iteration kernel
CASES = [(600, 560, BC_DIRICHLET0, "circular"), (640, 512, BC_PERIODIC, "stream")]

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2307_12276_gb300 as ad
from workloads import small_problem
nx, ny, bc, kind = {case!r}
p = small_problem(nx, ny, bc, kind, adv=(0.1, -0.05), dt_factor=200.0, s=2, c=(1 / 3, 2 / 3))
D = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda:0")
g = p.grid
op = ad.create_operator(nx, ny, bc, D(p.Dxx), D(p.Dxy), D(p.Dyy), 0.1, -0.05, ad.FP64)
v = D(np.random.default_rng(3).standard_normal(g.n))
stats, arrays = {{}}, {{}}
for key, kw in (("f9", dict(force_iters=9)), ("tol", dict(tol=1e-10))):
    out = torch.empty_like(v)
    ad.time_series(op)
    stats[key] = ad.leja_phi1(op, v, out, p.dt, **kw)
    stats[key + "_path"] = ad.series_timing(op)["kernel"]
    arrays[key] = out.cpu().numpy()
src = ad.Source([D(gk) for gk in p.source.g], list(p.source.h))
for s, c in ((1, (0.5,)), (2, (1 / 3, 2 / 3))):
    u = D(p.u0)
    stats["step%d" % s] = ad.expquad_step(op, u, 0.1, p.dt, s, c, src, tol=1e-10)
    arrays["step%d" % s] = u.cpu().numpy()
np.savez({prefix!r}, **arrays)
print(json.dumps(stats))
"""


def _run(case, prefix, env_extra):
    env = dict(os.environ)
    env.pop("AD_F64_NORMS", None)
    env.update(env_extra)
    code = CHILD.format(root=ROOT, case=case, prefix=prefix)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(prefix + ".npz")


@pytest.mark.parametrize("case", CASES)
def test_norm_squares_off_fp64_pipe_equal_fp64_fma_sums(case, tmp_path):
    """Forced and adaptive phi_1 actions and one- and two-stage steps on the
    per-iteration kernel with both ways of forming the norms: identical
    vectors and counts, error estimates to 1e-12."""
    need_gpu()
    sq, a_sq = _run(case, str(tmp_path / "sq"), {})
    fm, a_fm = _run(case, str(tmp_path / "fma"), {"AD_F64_NORMS": "fp64"})
    for key in ("f9", "tol"):
        assert sq[key + "_path"] == fm[key + "_path"] == "graph loop of per-iteration kernels"
    assert sq["f9"]["iters"] == 9
    for key in a_fm.files:
        assert sq[key]["iters"] == fm[key]["iters"], (key, sq[key], fm[key])
        assert sq[key]["converged"] and fm[key]["converged"], key
        assert sq[key]["err_est"] == pytest.approx(fm[key]["err_est"], rel=1e-12), key
        assert np.array_equal(a_sq[key], a_fm[key]), key


def test_power_of_two_scaling_and_oracle_estimate():
    """phi_1 of v, 2^400 v and 2^-400 v on the per-iteration kernel: the
    results scale exactly, the counts and the error estimates are the same;
    the estimate of a forced series equals the oracle's FP64 one to 1e-12, and
    the adaptive series matches the oracle (equal counts, or the borderline
    rule of gpu_util.oracle_at_gpu_count)."""
    need_gpu()
    p = small_problem(600, 560, BC_DIRICHLET0, "circular", adv=(0.1, -0.05), dt_factor=200.0)
    A, alpha = oracle_operator(p)
    op = ad().create_operator(600, 560, BC_DIRICHLET0, dev64(p.Dxx), dev64(p.Dxy), dev64(p.Dyy),
                              0.1, -0.05, ad().FP64)
    ad().set_spectral_bound(op, alpha)
    v = np.random.default_rng(11).standard_normal(p.grid.n)
    runs = {}
    for k in (0, 400, -400):
        for key, kw in (("f9", dict(force_iters=9)), ("tol", dict(tol=1e-10))):
            out = torch.empty(p.grid.n, dtype=torch.float64, device="cuda:0")
            ad().time_series(op)
            st = ad().leja_phi1(op, dev64(np.ldexp(v, k)), out, p.dt, **kw)
            assert ad().series_timing(op)["kernel"] == "graph loop of per-iteration kernels"
            runs[(k, key)] = (st, np.ldexp(out.cpu().numpy(), -k))
    for key in ("f9", "tol"):
        st0, out0 = runs[(0, key)]
        for k in (400, -400):
            st, out = runs[(k, key)]
            assert st["iters"] == st0["iters"] and st["converged"], (k, key)
            assert st["err_est"] == st0["err_est"], (k, key)
            assert np.array_equal(out, out0), (k, key)
    _, ost = leja.leja_phi1(A, v, p.dt, alpha, force_iters=9)
    assert runs[(0, "f9")][0]["err_est"] == pytest.approx(ost.err_est, rel=1e-12)
    st, out = runs[(0, "tol")]
    ref, ost = leja.leja_phi1(A, v, p.dt, alpha, tol=1e-10)

    def forced(k):
        r, s = leja.leja_phi1(A, v, p.dt, alpha, force_iters=k)
        return r, s.err_est
    alt = oracle_at_gpu_count(st["iters"], ost.iters, forced, 1e-10)
    assert_close(out, ref if alt is None else alt, 1e-11)
    if alt is None:
        assert st["err_est"] == pytest.approx(ost.err_est, rel=1e-12)


MOM_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_2307_12276_gb300 as ad
from workloads.fields import BC_DIRICHLET0
from workloads.momentum import momentum_problem
D = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device="cuda:0")
mp = momentum_problem(96, 80, 8, BC_DIRICHLET0, "circular", adv=(0.1, 0.05), dt_factor=100.0)
s = mp.spatial
op = ad.create_momentum_operator(96, 80, BC_DIRICHLET0, D(s.Dxx), D(s.Dxy), D(s.Dyy), mp.mom.P,
                                 mp.mom.beta, mp.mom.dpp, mp.mom.b, mp.mom.loss, ax=s.ax, ay=s.ay)
ad.momentum_spectral_bound(op)
v = D(mp.S.ravel() + 0.1 * np.random.default_rng(5).standard_normal(mp.S.size))
stats, arrays = {{}}, {{}}
for key, kw in (("f17", dict(force_iters=17)), ("tol", dict(tol=1e-10))):
    out = torch.empty_like(v)
    stats[key] = ad.momentum_leja_phi1(op, v, out, mp.dt, **kw)
    arrays[key] = out.cpu().numpy()
np.savez({prefix!r}, **arrays)
print(json.dumps(stats))
"""


def test_momentum_norm_squares_equal_fp64_fma_sums(tmp_path):
    """The momentum-coupled iteration with both ways of forming the norms:
    identical vectors and counts, error estimates to 1e-12."""
    need_gpu()
    res = {}
    for tag, env_extra in (("sq", {}), ("fma", {"AD_F64_NORMS": "fp64"})):
        env = dict(os.environ)
        env.pop("AD_F64_NORMS", None)
        env.update(env_extra)
        prefix = str(tmp_path / tag)
        code = MOM_CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), prefix=prefix)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[tag] = (json.loads(r.stdout.strip().splitlines()[-1]), np.load(prefix + ".npz"))
    (sq, a_sq), (fm, a_fm) = res["sq"], res["fma"]
    for key in a_fm.files:
        assert sq[key]["iters"] == fm[key]["iters"] and sq[key]["converged"], key
        assert sq[key]["err_est"] == pytest.approx(fm[key]["err_est"], rel=1e-12), key
        assert np.array_equal(a_sq[key], a_fm[key]), key
