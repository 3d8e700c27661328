"""Pins of the oracle MLP: analytic gradients against central differences,
tanh' = 1 - tanh^2, and one Adam step computed by hand."""
import numpy as np

from oracle import mlp


def _setup(seed=0, n_in=21, h=16, n_out=2, B=7):
    rng = np.random.default_rng(seed)
    n = sum(int(np.prod(s)) for s in mlp.shapes(n_in, h, n_out))
    theta = rng.standard_normal(n) * 0.3
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal((B, n_out))
    return theta, X, T, n_in, h, n_out


def test_gradient_matches_central_differences():
    theta, X, T, n_in, h, n_out = _setup()
    loss, g = mlp.loss_and_grad(theta, X, T, n_in, h, n_out)
    rng = np.random.default_rng(1)
    # a sample of coordinates from every parameter block
    sizes = [int(np.prod(s)) for s in mlp.shapes(n_in, h, n_out)]
    starts = np.cumsum([0] + sizes[:-1])
    idx = np.concatenate([st + rng.choice(sz, size=min(sz, 6), replace=False)
                          for st, sz in zip(starts, sizes)])
    eps = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (mlp.loss_and_grad(tp, X, T, n_in, h, n_out)[0]
              - mlp.loss_and_grad(tm, X, T, n_in, h, n_out)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_forward_definition_and_loss():
    theta, X, T, n_in, h, n_out = _setup(h=3, B=2)
    W1, b1, W2, b2, W3, b3 = mlp.unflatten(theta, n_in, h, n_out)
    y, _ = mlp.forward(theta, X, n_in, h, n_out)
    for b in range(2):
        a1 = [np.tanh(sum(X[b, i] * W1[i, j] for i in range(n_in)) + b1[j]) for j in range(h)]
        a2 = [np.tanh(sum(a1[i] * W2[i, j] for i in range(h)) + b2[j]) for j in range(h)]
        out = [sum(a2[i] * W3[i, k] for i in range(h)) + b3[k] for k in range(n_out)]
        assert np.allclose(y[b], out, rtol=1e-14, atol=1e-14)
    loss, _ = mlp.loss_and_grad(theta, X, T, n_in, h, n_out)
    assert abs(loss - 0.5 * np.sum((y - T) ** 2) / 2) < 1e-14


def test_tanh_derivative():
    z = np.linspace(-3, 3, 101)
    fd = (np.tanh(z + 1e-7) - np.tanh(z - 1e-7)) / 2e-7
    assert np.max(np.abs(fd - (1 - np.tanh(z) ** 2))) < 1e-8


def test_adam_first_step_by_hand():
    theta = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    th, m, v = mlp.adam_step(theta, g, np.zeros(2), np.zeros(2), 1, lr=0.1)
    # first step: mhat = g, vhat = g^2, so the update is -lr * g / (|g| + eps)
    assert np.allclose(th, theta - 0.1 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
