"""NumPy FP64 reference of the spectral-bound predictor network (oracle).

The paper estimates the spectrum with Gershgorin discs (Section 2); the
learned form replaces that estimate by a small multilayer perceptron whose
training data come from the method itself.  This module is the plain
reference of the network the CUDA kernels train and evaluate:

    h1 = tanh(x W1 + b1),  h2 = tanh(h1 W2 + b2),  y = h2 W3 + b3
    loss = 1/(2 B) sum_{b, k} (y_bk - t_bk)^2
    Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
          theta -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

Parameters are one flat vector in the order W1 (n_in x h), b1, W2 (h x h), b2,
W3 (h x n_out), b3, row-major.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss for
every parameter block, the tanh derivative, and one hand-computed Adam step.
"""
from __future__ import annotations

import numpy as np


def shapes(n_in: int, h: int, n_out: int):
    return [(n_in, h), (h,), (h, h), (h,), (h, n_out), (n_out,)]


def unflatten(theta, n_in, h, n_out):
    out, k = [], 0
    for s in shapes(n_in, h, n_out):
        size = int(np.prod(s))
        out.append(np.asarray(theta[k:k + size], dtype=np.float64).reshape(s))
        k += size
    return out


def forward(theta, X, n_in, h, n_out):
    W1, b1, W2, b2, W3, b3 = unflatten(theta, n_in, h, n_out)
    z1 = X @ W1 + b1
    a1 = np.tanh(z1)
    z2 = a1 @ W2 + b2
    a2 = np.tanh(z2)
    y = a2 @ W3 + b3
    return y, (X, a1, a2)


def loss_and_grad(theta, X, T, n_in, h, n_out):
    """Loss and its gradient with respect to the flat parameter vector."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    W1, b1, W2, b2, W3, b3 = unflatten(theta, n_in, h, n_out)
    y, (X, a1, a2) = forward(theta, X, n_in, h, n_out)
    r = y - T
    loss = 0.5 * float(np.sum(r * r)) / B
    dy = r / B
    gW3 = a2.T @ dy
    gb3 = dy.sum(axis=0)
    da2 = dy @ W3.T
    dz2 = da2 * (1.0 - a2 * a2)
    gW2 = a1.T @ dz2
    gb2 = dz2.sum(axis=0)
    da1 = dz2 @ W2.T
    dz1 = da1 * (1.0 - a1 * a1)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g


def adam_step(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba); t is the 1-based step count."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
