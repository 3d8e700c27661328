"""Learned spectral bound for the batched form: the driver around the library.

Section 2 of the paper bounds the spectrum with Gershgorin discs before every
Leja series.  Here a small network (``MLP``, kernels in csrc/mlp.cu) predicts
the bound and the iteration count from 21 per-field features, trained on
spectra the method itself computes (power iteration on generated fields).
Inside a batch the predicted bound replaces the power-iteration pass; a slice
whose series does not converge falls back to power iteration.

Every numerical step runs in the library: the features (recorded by
ad_create_operator), the training labels (ad_bound_training_sample), training
(ad_mlp_train), inference and the bound it implies (ad_learned_bounds).  This
module only generates the seeded training fields (workloads) and sequences
the calls.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

from . import (BC_DIRICHLET0, BC_PERIODIC, BOUND_POWER, FP64, MLP, batch_bind,
               batch_iteration_hint, batch_step, bound_training_sample, create_operator,
               expquad_step, learned_bounds, spectral_bound)

# training-field sides and their weights: every side class contributes about
# the same number of cells, so large grids are rare but present
TRAIN_SIDES = (64, 128, 256, 512, 1024, 2048)


def draw_side(rng: np.random.Generator, sides: Sequence[int] = TRAIN_SIDES) -> int:
    w = 1.0 / np.asarray(sides, dtype=np.float64)
    return int(rng.choice(np.asarray(sides), p=w / w.sum()))


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


def field_job(seed: int, k: int, sides: Sequence[int] = TRAIN_SIDES):
    """Field k of the training set of ``seed`` (independent of every other k)."""
    rng = np.random.default_rng([seed, k])
    return random_field(rng, draw_side(rng, sides))


def label_field(g, Dxx, Dxy, Dyy, ax, ay, dt, device, seed=0, power_iters=60, tol=1e-6):
    """Inputs and targets of one field (ad_bound_training_sample on an FP64
    operator of the field): returns (x[21], t[2], power-iteration |alpha|)."""
    import torch
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=device)
    op = create_operator(g.nx, g.ny, g.bc, T(Dxx), T(Dxy), T(Dyy), ax, ay, FP64)
    try:
        return bound_training_sample(op, dt, seed, power_iters=power_iters, safety=1.1, tol=tol)
    finally:
        op.close()


def build_dataset(n: int, seed: int, device, sides: Sequence[int] = TRAIN_SIDES,
                  workers: int = 0):
    """n labelled fields.  With workers > 1 the host-side field generation
    runs in a spawned process pool beside the GPU labelling."""
    xs, ts = [], []
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(field_job, seed, k, tuple(sides)) for k in range(n)]
            for k, f in enumerate(futs):
                x, t, _ = label_field(*f.result(), device=device, seed=seed * 100003 + k)
                futs[k] = None
                xs.append(x)
                ts.append(t)
    else:
        for k in range(n):
            x, t, _ = label_field(*field_job(seed, k, sides), device=device,
                                  seed=seed * 100003 + k)
            xs.append(x)
            ts.append(t)
    return np.stack(xs).astype(np.float32), np.stack(ts).astype(np.float32)


def train_bound_model(X, Y, device, epochs=3000, lr=3e-3, seed=0, hidden=64) -> MLP:
    import torch
    m = MLP(X.shape[1], hidden, Y.shape[1], seed=seed)
    m.train(torch.as_tensor(X, device=device), torch.as_tensor(Y, device=device), epochs=epochs,
            lr=lr, fit_normalization=True)
    return m


def predict_bounds(model: MLP, ops, dt, margin=1.1, bf16=True, batch=None):
    """Every operator's bound from the model (ad_learned_bounds, which also
    sets it); returns (alphas, predicted iterations).  With a batch of these
    operators, the predicted iteration counts also set its queue order
    (ad_batch_iteration_hint: the longest series first in every pass)."""
    alpha, iters = learned_bounds(model, ops, dt, margin=margin, bf16=bf16)
    if batch is not None:
        batch_iteration_hint(batch, iters)
    return alpha, iters


def batched_step_with_fallback(batch, ops, us, t, dt, sources, tol, power_iters=40):
    """One batched midpoint step.  A slice whose series did not converge keeps
    its input state (the batched step leaves it untouched); it then gets a
    power-iteration bound and repeats its step alone.  The batch is bound to
    the lists us and sources (ad_batch_bind) the first time they are passed,
    and stepped through the binding.  Returns (per-slice stats, list of
    fallback slice indices)."""
    bound = getattr(batch, "_bound", None)
    if bound is None or bound[0] is not us or bound[1] is not sources:
        batch_bind(batch, us, sources)
    st = batch_step(batch, t, dt, tol=tol, raise_not_converged=False)
    bad = [s for s in range(len(us)) if not st[s]["converged"]]
    for s in bad:
        spectral_bound(ops[s], BOUND_POWER, seed=s + 1, power_iters=power_iters, safety=1.1)
        st[s] = expquad_step(ops[s], us[s], t, dt, 1, (0.5,),
                             sources[s] if sources is not None else None, tol=tol)
    return st, bad
