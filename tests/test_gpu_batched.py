"""Batched exponential-midpoint step (one graph launch for many slices of
uneven size) against the FP64 oracle, slice by slice.

Each slice is an FP32-storage operator; the bar is the FP32 one (1e-5
relative L2).  Forced iteration counts make the comparison exact in method;
the adaptive case checks each slice's own stopping decision against the
oracle's.  The autotuner's JSON cache is checked for a round trip.
"""
import json
import os

import numpy as np
import pytest

from gpu_util import ad, devT, dev64, need_gpu, torch, assert_close
from oracle import integrators
from oracle import operator as oop
from oracle import spectral
from workloads import Grid, cell_centres, gaussian, tensor_from_b, b_circular
from workloads.fields import BC_DIRICHLET0

pytestmark = pytest.mark.gpu

SIZES = [(40, 33), (64, 64), (300, 70), (17, 23), (256, 256), (513, 40)]
# every nx % 4 == 0: the batch runs the warp-tile ring iteration kernel
SIZES_RING = [(40, 33), (64, 64), (300, 70), (4, 9), (256, 256), (516, 40), (128, 1)]


def _slice(nx, ny, dpar):
    g = Grid(nx, ny, BC_DIRICHLET0)
    X, Y = cell_centres(g)
    bx, by, w = b_circular(X, Y, 0.05)
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, dpar, 1e-3 * dpar, w)
    src = gaussian(X, Y, 0.0, 0.0, 0.1)
    u0 = gaussian(X, Y, 0.1, -0.1, 0.2)
    return g, Dxx, Dxy, Dyy, src, u0


def _build(autotune=False, sizes=None):
    slices, ops = [], []
    for k, (nx, ny) in enumerate(sizes or SIZES):
        g, Dxx, Dxy, Dyy, src, u0 = _slice(nx, ny, 1.0 + 3.0 * k)
        A = oop.assemble(g, Dxx, Dxy, Dyy, 0.05, 0.0)
        alpha = spectral.gershgorin(A)
        op = ad().create_operator(nx, ny, g.bc, dev64(Dxx), dev64(Dxy), dev64(Dyy), 0.05, 0.0,
                                  ad().FP32_STORAGE)
        ad().set_spectral_bound(op, alpha)
        slices.append((g, A, alpha, src, u0))
        ops.append(op)
    return slices, ops, ad().create_batch(ops, autotune=autotune)


def _dt(slices):
    # largest dt keeping every slice at gamma dt <= 150 (one substep)
    return min(150.0 / (-alpha / 4.0) for (_, _, alpha, _, _) in slices)


@pytest.mark.parametrize("force", [1, 20])
def test_batched_forced_matches_oracle(force):
    need_gpu()
    slices, ops, batch = _build()
    dt = _dt(slices)
    us = [devT(s[4], 1) for s in slices]
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, force_iters=force)
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        ref, ost = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                            lambda t, src=src: src.ravel(), alpha,
                                            force_iters=force)
        assert st[k]["iters"] == force
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, SIZES[k])))


def test_batched_adaptive_matches_oracle_per_slice():
    need_gpu()
    slices, ops, batch = _build()
    dt = _dt(slices)
    us = [devT(s[4], 1) for s in slices]
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6)
    iters = [s["iters"] for s in st]
    assert len(set(iters)) > 1                  # slices really stop at different counts
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        ref, ost = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                            lambda t, src=src: src.ravel(), alpha, tol=1e-10)
        _, ost6 = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                           lambda t, src=src: src.ravel(), alpha, tol=1e-6)
        assert abs(st[k]["iters"] - ost6.iters) <= 2, (k, st[k]["iters"], ost6.iters)
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, SIZES[k])))
    # a second step from the new state still matches (state reuse, cached scalars)
    u1 = [u.clone() for u in us]
    ad().batch_midpoint_step(batch, u1, dt, dt, srcs, tol=1e-6)
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        ref, _ = integrators.expquad_step(A, us[k].cpu().numpy().astype(np.float64), dt, dt, 1,
                                          (0.5,), lambda t, src=src: src.ravel(), alpha, tol=1e-10)
        assert_close(u1[k].cpu().numpy(), ref, 1e-5)


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    need_gpu()
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("AD_AUTOTUNE_CACHE", str(cache))
    _, _, b1 = _build(autotune=True)
    info1 = ad().batch_info(b1)
    data = json.loads(cache.read_text())
    assert len(data) == 1
    entry = next(iter(data.values()))
    assert entry["ty"] == info1["tile_rows"] and entry["ty"] in (8, 16, 32, 64, 128)
    assert entry["march"] == info1["marching"] and entry["march"] in (0, 1, 2)
    _, _, b2 = _build(autotune=True)            # served from the cache
    info2 = ad().batch_info(b2)
    assert info2["tile_rows"] == info1["tile_rows"]
    assert info2["marching"] == info1["marching"]
    assert abs(info2["tuned_ms"] - entry["ms"]) < 1e-6


def test_unconverged_slice_keeps_its_state():
    """A slice whose series cannot converge (a NaN in its state makes the norms
    non-finite) is left exactly as it was, the others advance as usual and the
    step reports NotConverged."""
    need_gpu()
    slices, ops, batch = _build()
    dt = _dt(slices)
    bad = 2
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]

    def states():
        us = [devT(s[4], 1) for s in slices]
        us[bad][5] = float("nan")
        return us

    us = states()
    before = us[bad].clone()
    with pytest.raises(ad().NotConverged):
        ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6)
    assert torch.equal(us[bad].view(torch.int32), before.view(torch.int32))
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        if k == bad:
            continue
        ref, _ = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, src=src: src.ravel(), alpha, tol=1e-10)
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, SIZES[k])))
    # the same call without raising gives the flag per slice
    us = states()
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6, raise_not_converged=False)
    assert [s["converged"] for s in st] == [k != bad for k in range(len(slices))]
    assert torch.equal(us[bad].view(torch.int32), before.view(torch.int32))


@pytest.mark.parametrize("force", [1, 17])
def test_ring_batch_forced_matches_oracle(force):
    """All slices 16-byte aligned: the warp-tile ring kernel runs the iterations."""
    need_gpu()
    slices, ops, batch = _build(sizes=SIZES_RING)
    dt = _dt(slices)
    us = [devT(s[4], 1) for s in slices]
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, force_iters=force)
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        ref, _ = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, src=src: src.ravel(), alpha,
                                          force_iters=force)
        assert st[k]["iters"] == force
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, SIZES_RING[k])))


def test_ring_batch_adaptive_and_tuned(tmp_path, monkeypatch):
    need_gpu()
    monkeypatch.setenv("AD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    slices, ops, batch = _build(autotune=True, sizes=SIZES_RING)
    info = ad().batch_info(batch)
    assert info["tile_rows"] in (16, 32, 64, 128)
    dt = _dt(slices)
    us = [devT(s[4], 1) for s in slices]
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6)
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        ref, _ = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, src=src: src.ravel(), alpha, tol=1e-10)
        _, ost6 = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                           lambda t, src=src: src.ravel(), alpha, tol=1e-6)
        assert abs(st[k]["iters"] - ost6.iters) <= 2, (k, st[k]["iters"], ost6.iters)
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, SIZES_RING[k])))


# every nx % 4 == 0 and ny >= 2: the two-iteration kernel (batch_pair_k)
SIZES_PAIR = [(40, 33), (64, 64), (300, 70), (4, 9), (256, 256), (516, 40), (124, 2)]


@pytest.mark.parametrize("force", [1, 2, 7, 20])
def test_pair_batch_forced_matches_oracle(force):
    """Odd counts stop after the first iteration of a launch; even counts leave
    d_m y_m to the flush kernel."""
    need_gpu()
    slices, ops, batch = _build(sizes=SIZES_PAIR)
    dt = _dt(slices)
    us = [devT(s[4], 1) for s in slices]
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, force_iters=force)
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        ref, _ = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, src=src: src.ravel(), alpha,
                                          force_iters=force)
        assert st[k]["iters"] == force
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, SIZES_PAIR[k])))


def test_pair_batch_adaptive_and_unconverged_slice():
    need_gpu()
    slices, ops, batch = _build(sizes=SIZES_PAIR)
    dt = _dt(slices)
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
    us = [devT(s[4], 1) for s in slices]
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6)
    for k, (g, A, alpha, src, u0) in enumerate(slices):
        ref, _ = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, src=src: src.ravel(), alpha, tol=1e-10)
        _, ost6 = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                           lambda t, src=src: src.ravel(), alpha, tol=1e-6)
        assert abs(st[k]["iters"] - ost6.iters) <= 2, (k, st[k]["iters"], ost6.iters)
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, SIZES_PAIR[k])))
    bad = 1
    us = [devT(s[4], 1) for s in slices]
    us[bad][5] = float("nan")
    before = us[bad].clone()
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6, raise_not_converged=False)
    assert [s["converged"] for s in st] == [k != bad for k in range(len(slices))]
    assert torch.equal(us[bad].view(torch.int32), before.view(torch.int32))


PAIR_CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import test_gpu_batched as tb
from gpu_util import ad, devT
slices, ops, batch = tb._build(sizes=tb.SIZES_PAIR)
dt = tb._dt(slices)
srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
out, stats = {{}}, {{}}
for key, kw in (("f7", dict(force_iters=7)), ("f8", dict(force_iters=8)), ("tol", dict(tol=1e-6))):
    us = [devT(s[4], 1) for s in slices]
    st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, **kw)
    stats[key] = [s["iters"] for s in st]
    stats["launches_" + key] = st[0]["kernel_launches"]
    for k, u in enumerate(us):
        out["%s_%d" % (key, k)] = u.cpu().numpy()
np.savez({prefix!r}, **out)
print(json.dumps(stats))
"""


@pytest.mark.parametrize("march", ["1", "2"])
def test_pair_batch_equals_ring_batch(tmp_path, march):
    """The two-iteration batch kernel, with either marching the autotuner
    chooses from (scalar or packed FP32 pair arithmetic), forms every entry
    as the one-iteration ring kernel does (AD_F32_PAIR=0): with equal counts,
    identical results."""
    need_gpu()
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for tag, env_extra in (("pair", {"AD_F32_MARCH": march}), ("ring", {"AD_F32_PAIR": "0"})):
        env = dict(os.environ)
        env.update(env_extra)
        env["AD_AUTOTUNE_CACHE"] = str(tmp_path / f"tune_{tag}.json")
        prefix = str(tmp_path / tag)
        code = PAIR_CHILD.format(root=root, tests=os.path.join(root, "tests"), prefix=prefix)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[tag] = (json.loads(r.stdout.strip().splitlines()[-1]), np.load(prefix + ".npz"))
    (sp, ap), (sr, ar) = res["pair"], res["ring"]
    assert {k: v for k, v in sp.items() if not k.startswith("launches")} == \
        {k: v for k, v in sr.items() if not k.startswith("launches")}
    for key in ar.files:
        assert np.array_equal(ap[key], ar[key]), key


def test_persistent_batch_equals_graph_loop(tmp_path):
    """The whole series of every slice in one persistent cooperative launch
    (each slice's pass waiting only for its own previous pass) against the
    graph loop of two-iteration launches (AD_BATCH_PERSIST=0): the same tiles
    and the same order of every sum, so identical counts and results; the
    persistent step is three kernels (start, series, finish)."""
    need_gpu()
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for tag, env_extra in (("persist", {}), ("loop", {"AD_BATCH_PERSIST": "0"})):
        env = dict(os.environ)
        env.update(env_extra)
        env["AD_AUTOTUNE_CACHE"] = str(tmp_path / f"tune_{tag}.json")
        prefix = str(tmp_path / tag)
        code = PAIR_CHILD.format(root=root, tests=os.path.join(root, "tests"), prefix=prefix)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[tag] = (json.loads(r.stdout.strip().splitlines()[-1]), np.load(prefix + ".npz"))
    (sp, ap), (sl, al) = res["persist"], res["loop"]
    for key in ("f7", "f8", "tol"):
        assert sp[key] == sl[key], key
        assert sp["launches_" + key] == 3 < sl["launches_" + key], key
    for key in al.files:
        assert np.array_equal(ap[key], al[key]), key


def test_queue_order_follows_iterations_and_changes_no_result():
    """ad_batch_iteration_hint queues the slices expected to iterate longest
    first; after each step the batch re-queues them by that step's counts
    (decreasing, ties in slice order); the queue order changes no result (each
    slice's tile sums keep their order), whatever it is."""
    need_gpu()
    slices, ops, batch = _build(sizes=SIZES_PAIR)
    dt = _dt(slices)
    srcs = [ad().Source([devT(s[3], 1)], None) for s in slices]
    S = len(slices)
    ad().batch_iteration_hint(batch, None)
    assert ad().batch_order(batch) == list(range(S))
    us0 = [devT(s[4], 1) for s in slices]
    st0 = ad().batch_midpoint_step(batch, us0, 0.0, dt, srcs, tol=1e-6)
    iters = [s["iters"] for s in st0]
    assert len(set(iters)) > 1                  # the slices need different counts
    assert ad().batch_order(batch) == sorted(range(S), key=lambda k: -iters[k])
    for hint in (list(range(S)), [float((7 * k) % S) for k in range(S)]):
        ad().batch_iteration_hint(batch, hint)
        assert ad().batch_order(batch) == sorted(range(S), key=lambda k: -hint[k])
        us = [devT(s[4], 1) for s in slices]
        st = ad().batch_midpoint_step(batch, us, 0.0, dt, srcs, tol=1e-6)
        assert [s["iters"] for s in st] == iters
        for k in range(S):
            assert torch.equal(us[k].view(torch.int32), us0[k].view(torch.int32)), (hint, k)
    with pytest.raises(ad().AdError):
        ad().batch_iteration_hint(batch, [float("nan")] * S)
    with pytest.raises(ValueError):
        ad().batch_iteration_hint(batch, [1.0] * (S + 1))


def test_bound_step_equals_midpoint_step():
    """ad_batch_bind + ad_batch_step give ad_batch_midpoint_step's results bit
    for bit (time-dependent sources included, their profiles evaluated at each
    step's midpoint); stepping an unbound batch is refused; a rebind moves the
    step to other vectors."""
    need_gpu()
    slices, ops, batch = _build(sizes=SIZES_PAIR)
    dt = _dt(slices)
    prof = [lambda t: 1.0 + 0.5 * np.sin(2.0 * np.pi * t)]
    srcs = [ad().Source([devT(s[3], 1)], prof) for s in slices]
    with pytest.raises(ad().AdError):
        ad().batch_step(batch, 0.0, dt)
    ua = [devT(s[4], 1) for s in slices]
    ub = [devT(s[4], 1) for s in slices]
    sa, sb = [], []
    for k in range(3):
        sa.append(ad().batch_midpoint_step(batch, ua, k * dt, dt, srcs, tol=1e-6))
    ad().batch_bind(batch, ub, srcs)
    for k in range(3):
        sb.append(ad().batch_step(batch, k * dt, dt, tol=1e-6))
    assert [[s["iters"] for s in st] for st in sa] == [[s["iters"] for s in st] for st in sb]
    for x, y in zip(ua, ub):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    uc = [devT(s[4], 1) for s in slices]
    ad().batch_bind(batch, uc, srcs)
    ad().batch_step(batch, 0.0, dt, tol=1e-6)
    assert not torch.equal(uc[0], devT(slices[0][4], 1))
    assert torch.equal(ub[0].view(torch.int32), ua[0].view(torch.int32))   # untouched by the rebind
