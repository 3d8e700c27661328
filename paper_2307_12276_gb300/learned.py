"""Learned spectral bound for the batched form.

Section 2 of the paper bounds the spectrum with Gershgorin discs before every
Leja series.  Here a small network (``MLP``, kernels in csrc/mlp.cu) predicts
the bound and the iteration count from 21 per-field features, trained on
spectra the method itself computes (power iteration on generated fields).
Inside a batch the predicted bound replaces the power-iteration pass; a slice
whose series does not converge falls back to power iteration.

Targets are dimensionless so that a model trained on small generated grids
serves large slices:  t0 = log(|alpha| dx^2 / D_par),  t1 = log(iterations).

Every numerical step runs in the library's kernels; this module only drives
them (field generation for training uses the seeded input generators).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import (BC_DIRICHLET0, BC_PERIODIC, BOUND_POWER, FP64, MLP, NotConverged,
               batch_midpoint_step, create_operator, expquad_step, field_features, leja_phi1,
               set_spectral_bound, spectral_bound)


@dataclass
class FieldSample:
    features: np.ndarray      # 21 inputs
    targets: np.ndarray       # (t0, t1)
    alpha: float              # power-iteration bound used as the label


def random_field(rng: np.random.Generator, side: int):
    """One generated training field: random stream-function / circular /
    uniform direction field, D_par in [1, 100], D_perp / D_par in [1e-6, 1e-2],
    |a| in [0, 1], dt in [10, 1000] Delta t_CFL (log-uniform draws)."""
    from workloads import (Grid, b_circular, b_stream, b_uniform, cell_centres, cfl_dt,
                           tensor_from_b)
    g = Grid(side, side, BC_DIRICHLET0 if rng.random() < 0.7 else BC_PERIODIC)
    X, Y = cell_centres(g)
    kind = rng.integers(3)
    dpar = 10 ** rng.uniform(0.0, 2.0)
    dperp = dpar * 10 ** rng.uniform(-6.0, -2.0)
    if kind == 0:
        bx, by, w = b_stream(X, Y, int(rng.integers(1 << 30)))
    elif kind == 1:
        bx, by, w = b_circular(X, Y, 0.05)
    else:
        bx, by = b_uniform(X.shape, rng.uniform(0.0, 180.0))
        w = None
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, dpar, dperp, w)
    amag = rng.uniform(0.0, 1.0)
    ang = rng.uniform(0.0, 2 * math.pi)
    ax, ay = amag * math.cos(ang), amag * math.sin(ang)
    dt = 10 ** rng.uniform(1.0, 3.0) * cfl_dt(g, Dxx, Dxy, Dyy)
    return g, Dxx, Dxy, Dyy, ax, ay, dt


def label_field(g, Dxx, Dxy, Dyy, ax, ay, dt, device, seed=0, power_iters=60,
                tol=1e-6) -> FieldSample:
    """Features (GPU kernel), the power-iteration bound and the Leja iteration
    count of phi_1(dt A) v at ``tol`` with alpha = 1.1 x the estimate."""
    import torch
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=device)
    dxx, dxy, dyy = T(Dxx), T(Dxy), T(Dyy)
    amax = math.hypot(ax, ay)
    f = field_features(g.nx, g.ny, g.bc, dxx, dxy, dyy, amax, dt)
    op = create_operator(g.nx, g.ny, g.bc, dxx, dxy, dyy, ax, ay, FP64)
    a_est = -spectral_bound(op, BOUND_POWER, seed=seed + 1, power_iters=power_iters, safety=1.0)
    set_spectral_bound(op, -1.1 * a_est)
    v = torch.as_tensor(np.random.default_rng(seed).standard_normal(g.n), device=device)
    out = torch.empty_like(v)
    try:
        st = leja_phi1(op, v, out, dt, tol=tol)
        iters = st["iters"]
    except NotConverged as e:
        iters = e.stats["iters"] if e.stats else 500
    op.close()
    dx = min(g.dx, g.dy)
    t0 = math.log(a_est * dx * dx / math.exp(f[0]))
    return FieldSample(f, np.array([t0, math.log(max(iters, 1))], dtype=np.float32), -a_est)


def build_dataset(n: int, seed: int, device, sides: Sequence[int] = (32, 48, 64, 96)):
    rng = np.random.default_rng(seed)
    samples = []
    for k in range(n):
        side = int(rng.choice(np.asarray(sides)))
        samples.append(label_field(*random_field(rng, side), device=device, seed=seed * 100003 + k))
    X = np.stack([s.features for s in samples]).astype(np.float32)
    Y = np.stack([s.targets for s in samples]).astype(np.float32)
    return X, Y, samples


def train_bound_model(X, Y, device, epochs=3000, lr=3e-3, seed=0, hidden=64) -> MLP:
    import torch
    m = MLP(X.shape[1], hidden, Y.shape[1], seed=seed)
    m.train(torch.as_tensor(X, device=device), torch.as_tensor(Y, device=device), epochs=epochs,
            lr=lr, fit_normalization=True)
    return m


def predict_bounds(m: MLP, feats, dxs: Sequence[float], device, margin=1.1, bf16=True):
    """alpha_s = -margin * exp(t0) D_par / dx^2 and the predicted iterations.
    ``feats``: (S, 21) float32 array or device tensor."""
    import torch
    X = torch.as_tensor(feats, device=device, dtype=torch.float32).contiguous()
    pred = m.predict(X, bf16=bf16).double().cpu().numpy()
    dpar = np.exp(X[:, 0].double().cpu().numpy())
    dx = np.asarray(dxs, dtype=np.float64)
    alpha = -margin * np.exp(pred[:, 0]) * dpar / (dx * dx)
    return alpha, np.exp(pred[:, 1])


def batched_step_with_fallback(batch, ops, us, t, dt, sources, tol, power_iters=40):
    """One batched midpoint step.  A slice whose series did not converge keeps
    its input state (the batched step leaves it untouched); it then gets a
    power-iteration bound and repeats its step alone.  Returns (per-slice
    stats, list of fallback slice indices)."""
    st = batch_midpoint_step(batch, us, t, dt, sources, tol=tol, raise_not_converged=False)
    bad = [s for s in range(len(us)) if not st[s]["converged"]]
    for s in bad:
        spectral_bound(ops[s], BOUND_POWER, seed=s + 1, power_iters=power_iters, safety=1.1)
        st[s] = expquad_step(ops[s], us[s], t, dt, 1, (0.5,),
                             sources[s] if sources is not None else None, tol=tol)
    return st, bad
