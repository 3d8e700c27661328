"""The learned spectral bound: network kernels against the NumPy oracle
(gradients, training, BF16 inference), the feature kernel, and the learned
bound inside a batch with power-iteration fallback against the FP64 oracle."""
import math

import numpy as np
import pytest

from gpu_util import DEV, ad, dev64, devT, need_gpu, rel, torch
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


def test_learned_bound_in_batch_with_fallback():
    need_gpu()
    from paper_2307_12276_gb300 import learned
    X, Y, samples = learned.build_dataset(240, seed=11, device=DEV, sides=(32, 48, 64))
    model = learned.train_bound_model(X[:200], Y[:200], DEV, epochs=1500, lr=3e-3)
    # relative error of the predicted dimensionless bound on held-out fields
    pred = model.predict(torch.as_tensor(X[200:], device=DEV)).cpu().numpy()
    err = np.abs(np.exp(pred[:, 0] - Y[200:, 0]) - 1.0)
    assert np.median(err) < 0.15
    # a small batch: learned bound, fallback where needed, parity with the oracle
    slices, ops, us, srcs = [], [], [], []
    feats, dxs = [], []
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
        feats.append(ad().field_features(side, side, g.bc, dev64(Dxx), dev64(Dxy), dev64(Dyy), 0.05,
                                         1.0))
        dxs.append(g.dx)
    gam = max(-spectral.gershgorin(s[1]) / 4 for s in slices)
    dt = 100.0 / gam
    feats = np.stack(feats)
    feats[:, 4] = math.log(dt)
    alpha, _ = learned.predict_bounds(model, feats, dxs, DEV, margin=1.2)
    for op, a in zip(ops, alpha):
        ad().set_spectral_bound(op, float(a))
    batch = ad().create_batch(ops, autotune=False)
    st, fallback = learned.batched_step_with_fallback(batch, ops, us, 0.0, dt, srcs, tol=1e-6)
    assert all(s["converged"] for s in st)
    for k, (g, A, src, u0) in enumerate(slices):
        ref, _ = integrators.expquad_step(A, u0.ravel(), 0.0, dt, 1, (0.5,),
                                          lambda t, src=src: src.ravel(),
                                          spectral.gershgorin(A), tol=1e-10)
        assert rel(us[k].cpu().numpy(), ref) <= 1e-5, (k, fallback)
