"""The learned spectral bound: network kernels against the NumPy oracle
(gradients, training, BF16 inference), the feature kernel, and the learned
bound inside a batch with power-iteration fallback against the FP64 oracle."""
import math

import numpy as np
import pytest

from gpu_util import DEV, ad, dev64, devT, need_gpu, torch, assert_close
from oracle import integrators, mlp as omlp
from oracle import operator as oop
from oracle import spectral
from workloads import Grid, b_circular, b_uniform, cell_centres, gaussian, tensor_from_b
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC

pytestmark = pytest.mark.gpu


def test_mlp_gradient_matches_oracle():
    need_gpu()
    m = ad().MLP(21, 64, 2, seed=3)
    rng = np.random.default_rng(4)
    theta = (rng.standard_normal(m.n_params) * 0.2).astype(np.float32)
    m.set_params(theta)
    X = rng.standard_normal((300, 21)).astype(np.float32)
    Y = rng.standard_normal((300, 2)).astype(np.float32)
    L, g = m.loss_grad(torch.as_tensor(X, device=DEV), torch.as_tensor(Y, device=DEV))
    Lr, gr = omlp.loss_and_grad(theta.astype(np.float64), X.astype(np.float64),
                                Y.astype(np.float64), 21, 64, 2)
    assert abs(L - Lr) <= 1e-5 * abs(Lr)
    assert np.linalg.norm(g - gr) <= 1e-5 * np.linalg.norm(gr)


def test_mlp_training_and_bf16_inference():
    need_gpu()
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (2000, 21)).astype(np.float32)
    Y = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2], np.exp(0.5 * X[:, 3])], 1).astype(np.float32)
    Xd, Yd = torch.as_tensor(X, device=DEV), torch.as_tensor(Y, device=DEV)
    m = ad().MLP(21, 64, 2, seed=1)
    L0 = m.loss_grad(Xd, Yd)[0]
    L = m.train(Xd, Yd, epochs=1500, lr=3e-3)
    assert L < 0.05 * max(L0, 1.0)
    p32 = m.predict(Xd, bf16=False).cpu().numpy()
    p16 = m.predict(Xd, bf16=True).cpu().numpy()
    # the FP32 forward equals the oracle forward with the trained parameters
    xm, xs, ym, ys = m.normalization()
    ref, _ = omlp.forward(m.get_params().astype(np.float64), (X - xm) / xs, 21, 64, 2)
    assert np.max(np.abs(p32 - (ref * ys + ym))) <= 1e-4 * np.max(np.abs(p32))
    assert np.max(np.abs(p16 - p32)) <= 0.05 * np.max(np.abs(p32))


def test_field_features_uniform_and_circular():
    need_gpu()
    g = Grid(64, 64, BC_PERIODIC)
    X, Y = cell_centres(g)
    bx, by = b_uniform(X.shape, 30.0)
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, 4.0, 1e-3)
    f = ad().field_features(64, 64, 0, dev64(Dxx), dev64(Dxy), dev64(Dyy), 0.5, 1e-3)
    assert abs(math.exp(f[0]) - 4.0) < 1e-4 and abs(math.exp(f[1]) - 1e-3) < 1e-6
    assert abs(f[2] - math.log(0.5 + 1e-6)) < 1e-6 and abs(f[3] - math.log(2 / 64)) < 1e-6
    hist = f[5:]
    assert abs(hist.sum() - 1.0) < 1e-5
    assert int(np.argmax(hist)) == int((math.radians(30.0) + math.pi / 2) / math.pi * 16)
    bx, by, w = b_circular(X, Y, 0.05)
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, 1.0, 1e-4, w)
    hist = ad().field_features(64, 64, 0, dev64(Dxx), dev64(Dxy), dev64(Dyy), 0.0, 1e-3)[5:]
    assert hist.max() < 0.15                  # circular directions spread over all bins


def _small_batch(model, margin=1.2):
    """Four FP32 slices of uneven size (circular field, constant advection)
    and the shared step 100 / max gamma (Gershgorin)."""
    slices, ops, us, srcs, fields = [], [], [], [], []
    for k, side in enumerate((40, 64, 96, 72)):
        g = Grid(side, side, BC_DIRICHLET0)
        Xc, Yc = cell_centres(g)
        bx, by, w = b_circular(Xc, Yc, 0.05)
        dpar = 1.0 + 5.0 * k
        Dxx, Dxy, Dyy = tensor_from_b(bx, by, dpar, 1e-3 * dpar, w)
        op = ad().create_operator(side, side, g.bc, dev64(Dxx), dev64(Dxy), dev64(Dyy), 0.05, 0.0,
                                  ad().FP32_STORAGE)
        A = oop.assemble(g, Dxx, Dxy, Dyy, 0.05, 0.0)
        src = gaussian(Xc, Yc, 0.0, 0.0, 0.1)
        u0 = gaussian(Xc, Yc, 0.1, -0.1, 0.2)
        slices.append((g, A, src, u0))
        ops.append(op)
        us.append(devT(u0, 1))
        srcs.append(ad().Source([devT(src, 1)], None))
        fields.append((Dxx, Dxy, Dyy))
    gam = max(-spectral.gershgorin(s[1]) / 4 for s in slices)
    return slices, ops, us, srcs, fields, 100.0 / gam


@pytest.fixture(scope="module")
def bound_model():
    need_gpu()
    from paper_2307_12276_gb300 import learned
    X, Y = learned.build_dataset(240, seed=11, device=DEV, sides=(32, 48, 64))
    model = learned.train_bound_model(X[:200], Y[:200], DEV, epochs=1500, lr=3e-3)
    return model, X, Y


def test_learned_bound_heldout(bound_model):
    """Relative error of the predicted dimensionless bound on held-out fields."""
    model, X, Y = bound_model
    pred = model.predict(torch.as_tensor(X[200:], device=DEV)).cpu().numpy()
    err = np.abs(np.exp(pred[:, 0] - Y[200:, 0]) - 1.0)
    assert np.median(err) < 0.15


def test_training_sample_against_oracle():
    """ad_bound_training_sample: its power estimate agrees with the oracle's
    power iteration from the same SplitMix64 start, its features with
    ad_field_features, and its targets follow from them."""
    need_gpu()
    from paper_2307_12276_gb300 import learned
    g, Dxx, Dxy, Dyy, ax, ay, dt = learned.field_job(5, 3, sides=(48,))
    op = ad().create_operator(g.nx, g.ny, g.bc, dev64(Dxx), dev64(Dxy), dev64(Dyy), ax, ay,
                              ad().FP64)
    x, t, est = ad().bound_training_sample(op, dt, seed=17, power_iters=60, safety=1.1, tol=1e-6)
    A = oop.assemble(g, Dxx, Dxy, Dyy, ax, ay)
    x0 = spectral.splitmix64_uniform(g.n, 18)
    a_ref, _ = spectral.power_iteration(A, x0, iters=60, safety=1.0)
    assert abs(est - (-a_ref)) <= 1e-10 * abs(a_ref)
    f = ad().field_features(g.nx, g.ny, g.bc, dev64(Dxx), dev64(Dxy), dev64(Dyy),
                            math.hypot(ax, ay), dt)
    assert np.allclose(x, f, rtol=1e-5, atol=1e-6)
    dx = min(g.dx, g.dy)
    assert abs(t[0] - math.log(est * dx * dx / math.exp(float(x[0])))) <= 1e-5
    assert ad().get_spectral_bound(op) == pytest.approx(-1.1 * est, rel=1e-15)
    op.close()


@pytest.mark.parametrize("bf16", [False, True])
def test_learned_bounds_through_capi(bound_model, bf16):
    """ad_learned_bounds against a NumPy restatement of its back-transform
    alpha = -margin exp(t0) D_par / dx^2 on the model's own predictions; the
    operators keep the bound; ad_spectral_bound(op, LEARNED) gives the same."""
    model = bound_model[0]
    slices, ops, us, srcs, fields, dt = _small_batch(model)
    margin = 1.2
    alpha, iters = ad().learned_bounds(model, ops, dt, margin=margin, bf16=bf16)
    feats = np.stack([ad().field_features(g.nx, g.ny, g.bc, dev64(D[0]), dev64(D[1]), dev64(D[2]),
                                          0.05, dt) for (g, _, _, _), D in zip(slices, fields)])
    pred = model.predict(torch.as_tensor(feats, device=DEV), bf16=bf16).double().cpu().numpy()
    dx = np.array([min(s[0].dx, s[0].dy) for s in slices])
    ref = -margin * np.exp(pred[:, 0]) * np.exp(feats[:, 0].astype(np.float64)) / dx ** 2
    tol = 2e-2 if bf16 else 1e-5
    assert np.allclose(alpha, ref, rtol=tol), (alpha, ref)
    assert np.allclose(iters, np.exp(pred[:, 1]), rtol=tol)
    for op, a in zip(ops, alpha):
        assert ad().get_spectral_bound(op) == a
    # ad_spectral_bound's learned method runs the BF16 inference
    a16, _ = ad().learned_bounds(model, [ops[1]], dt, margin=margin, bf16=True)
    ad().set_bound_model(ops[1], model, margin=margin, dt=dt)
    a1 = ad().spectral_bound(ops[1], ad().BOUND_LEARNED)
    assert a1 == pytest.approx(a16[0], rel=1e-12)
    ad().set_bound_model(ops[1], None)
    with pytest.raises(ad().AdError):
        ad().spectral_bound(ops[1], ad().BOUND_LEARNED)


@pytest.mark.parametrize("force_bad", [False, True])
def test_learned_bound_in_batch_with_fallback(bound_model, force_bad):
    """The learned bounds drive a batched step (and their iteration counts its
    queue order); with force_bad one slice's
    bound is cut to 0.02 x its Gershgorin bound, so the spectrum reaches far
    beyond the Leja interval and the series diverges (its FP32 terms overflow
    long before the stopping rule could hold): the fallback must list exactly
    that slice and still leave it matching the oracle."""
    from paper_2307_12276_gb300 import learned
    model = bound_model[0]
    slices, ops, us, srcs, fields, dt = _small_batch(model)
    batch = ad().create_batch(ops, autotune=False)
    alpha, it_pred = learned.predict_bounds(model, ops, dt, margin=1.2, batch=batch)
    # the predicted counts set the batch's queue order (longest series first)
    assert ad().batch_order(batch) == sorted(range(len(ops)), key=lambda k: -it_pred[k])
    bad = 2
    if force_bad:
        ad().set_spectral_bound(ops[bad], 0.02 * spectral.gershgorin(slices[bad][1]))
    st, fallback = learned.batched_step_with_fallback(batch, ops, us, 0.0, dt, srcs, tol=1e-6)
    assert fallback == ([bad] if force_bad else [])
    assert all(s["converged"] for s in st)
    for k, (g, A, src, u0) in enumerate(slices):
        ref, _ = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, src=src: src.ravel(),
                                          spectral.gershgorin(A), tol=1e-10)
        assert_close(us[k].cpu().numpy(), ref, 1e-5, str((k, fallback)))
