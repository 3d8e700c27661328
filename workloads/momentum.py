"""Inputs of the momentum-coupled transport problem of Eq. cr_full.

Only inputs: a spatial problem (``configs.small_problem`` fields or a named
config), logarithmic momentum faces, the per-cell scale beta_k of the spatial
diffusion, face values of D_pp and b = pdot - (p/3) div v, per-cell loss
rates, an initial field and a time-independent source on the (p, y, x) grid.
No discretisation and no time stepping happen here.

Physical shapes (synthetic, of the kind used for Galactic cosmic rays):
  * momentum 1 .. pmax (arbitrary units), log-spaced faces;
  * D(x, y, p) = (p / p0)^delta D(x, y) with delta = 0.5 (Kraichnan-like);
  * D_pp = kappa p^2 (reacceleration by a p-independent Alfven speed);
  * b = -zeta p^2 - (p / 3) div v (quadratic losses and adiabatic cooling for
    an expanding wind, div v > 0);
  * loss rate L = 1/tau_f + 1/tau_r constant;
  * source and initial field: a spatial Gaussian times a power law p^-2.2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .configs import Problem, small_problem
from .fields import BC_DIRICHLET0, cell_centres, cfl_dt, gaussian


@dataclass
class MomentumInputs:
    P: np.ndarray          # np + 1 faces
    beta: np.ndarray       # np spatial-diffusion scales
    dpp: np.ndarray        # np + 1 face values of D_pp
    b: np.ndarray          # np + 1 face values of pdot - (p/3) div v
    loss: np.ndarray       # np loss rates

    @property
    def np(self) -> int:
        return len(self.beta)


@dataclass
class MomentumProblem:
    spatial: Problem       # grid, D(x, y), constant advection
    mom: MomentumInputs
    u0: np.ndarray         # (np, ny, nx)
    S: np.ndarray          # (np, ny, nx), time-independent
    dt: float
    tol: float


def momentum_inputs(npm: int, pmax: float = 1e3, delta: float = 0.5, kappa: float = 20.0,
                    zeta: float = 0.05, divv: float = 30.0, loss: float = 2.0,
                    p0: float = 10.0) -> MomentumInputs:
    P = np.geomspace(1.0, pmax, npm + 1)
    pc = np.sqrt(P[:-1] * P[1:])
    return MomentumInputs(P=P, beta=(pc / p0) ** delta, dpp=kappa * P ** 2,
                          b=-zeta * P ** 2 - P / 3.0 * divv, loss=np.full(npm, loss))


def momentum_problem(nx: int, ny: int, npm: int, bc: int = BC_DIRICHLET0, kind: str = "circular",
                     seed: int = 11, adv=(0.0, 0.0), dt_factor: float = 100.0, tol: float = 1e-10,
                     **mom_kw) -> MomentumProblem:
    """A seeded coupled problem; dt = dt_factor x Delta t_CFL of the spatial
    operator at the largest beta_k."""
    sp_ = small_problem(nx, ny, bc, kind, seed=seed, adv=adv)
    mom = momentum_inputs(npm, **mom_kw)
    X, Y = cell_centres(sp_.grid)
    pc = np.sqrt(mom.P[:-1] * mom.P[1:])
    spectrum = pc ** -2.2
    blob = gaussian(X, Y, 0.2, -0.1, 0.2)
    rng = np.random.default_rng(seed + 1)
    u0 = spectrum[:, None, None] * (gaussian(X, Y, -0.1, 0.2, 0.3)[None]
                                    + 0.01 * rng.standard_normal((npm,) + X.shape))
    S = 5.0 * spectrum[:, None, None] * blob[None]
    bmax = float(np.max(mom.beta))
    cfl = cfl_dt(sp_.grid, bmax * sp_.Dxx, bmax * sp_.Dxy, bmax * sp_.Dyy)
    return MomentumProblem(spatial=sp_, mom=mom, u0=u0, S=S, dt=dt_factor * cfl, tol=tol)
