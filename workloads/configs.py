"""Workload descriptions: the five synthetic configurations and small test cases.

Each ``Problem`` carries everything both sides need: grid, coefficient fields,
advection (constant or a field), a separable source, the initial field, the
step size and count, the integrator and the tolerance.  Nothing here performs
a step of the method.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

from .fields import (BC_DIRICHLET0, BC_PERIODIC, Grid, SeparableSource, b_circular,
                     b_stream, b_uniform, cell_centres, cfl_dt, gaussian, tensor_from_b)


@dataclass
class Problem:
    name: str
    grid: Grid
    Dxx: np.ndarray
    Dxy: np.ndarray
    Dyy: np.ndarray
    ax: float = 0.0             # constant advection (used when ax_field is None)
    ay: float = 0.0
    ax_field: Optional[np.ndarray] = None
    ay_field: Optional[np.ndarray] = None
    source: SeparableSource = field(default_factory=SeparableSource)
    u0: Optional[np.ndarray] = None
    dt: float = 0.0
    steps: int = 1
    s: int = 1                   # stages of the exponential quadrature
    c: Tuple[float, ...] = (0.5,)
    tol: float = 1e-10
    cfl: float = 0.0

    def ax_arr(self):
        return self.ax_field if self.ax_field is not None else np.full_like(self.Dxx, self.ax)

    def ay_arr(self):
        return self.ay_field if self.ay_field is not None else np.full_like(self.Dxx, self.ay)

    def source_at(self, t: float) -> np.ndarray:
        out = np.zeros_like(self.Dxx)
        for gk, hk in zip(self.source.g, self.source.h):
            out += hk(t) * gk
        return out


def config0(nx: int = 64) -> Problem:
    """64^2 periodic FP64: uniform b at 30 deg, D_par 1, D_perp 1e-3, a = 0,
    constant Gaussian source (amp 1, sigma 0.1, origin), Gaussian u0 (sigma 0.2),
    exponential midpoint, tol 1e-10, dt = 100 Delta t_CFL, 10 steps."""
    g = Grid(nx, nx, BC_PERIODIC)
    X, Y = cell_centres(g)
    bx, by = b_uniform(X.shape, 30.0)
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, 1.0, 1e-3)
    src = SeparableSource([gaussian(X, Y, 0.0, 0.0, 0.1)], [lambda t: 1.0])
    cfl = cfl_dt(g, Dxx, Dxy, Dyy)
    return Problem("c0-64sq-periodic-uniform30-midpoint", g, Dxx, Dxy, Dyy, source=src,
                   u0=gaussian(X, Y, 0.0, 0.0, 0.2), dt=100.0 * cfl, steps=10, s=1,
                   c=(0.5,), tol=1e-10, cfl=cfl)


def config1(nx: int = 512, dt_factor: float = 200.0, steps: int = 1) -> Problem:
    """512^2 zero-Dirichlet FP64: circular b (isotropic blend r < 0.05), D_par 1,
    D_perp 1e-4, a = (0.1, 0.05), S = G(sigma 0.05 at (0.3, 0.3)) (1 + sin 2 pi t),
    two-stage exponential quadrature c = (1/3, 2/3), tol 1e-10,
    dt = dt_factor * Delta t_CFL with dt_factor in {50, 200, 1000}."""
    g = Grid(nx, nx, BC_DIRICHLET0)
    X, Y = cell_centres(g)
    bx, by, w = b_circular(X, Y, 0.05)
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, 1.0, 1e-4, w)
    src = SeparableSource([gaussian(X, Y, 0.3, 0.3, 0.05)],
                          [lambda t: 1.0 + float(np.sin(2.0 * np.pi * t))])
    cfl = cfl_dt(g, Dxx, Dxy, Dyy)
    return Problem(f"c1-{nx}sq-dirichlet-circular-expquad2-dt{int(dt_factor)}cfl", g,
                   Dxx, Dxy, Dyy, ax=0.1, ay=0.05, source=src,
                   u0=gaussian(X, Y, 0.0, 0.5, 0.1), dt=dt_factor * cfl, steps=steps, s=2,
                   c=(1.0 / 3.0, 2.0 / 3.0), tol=1e-10, cfl=cfl)


def config2(nx: int = 4096, seed: int = 0, tol: float = 1e-6, steps: int = 10) -> Problem:
    """4096^2 zero-Dirichlet: b from a random-phase 8-mode stream function
    (seed 0), D_par 1, D_perp = 10^U(-6, -2) (seed 1), a = 0, 16 Gaussian sources
    (sigma 0.02) at U(-0.9, 0.9)^2 (seed 2), Gaussian u0 (sigma 0.2),
    exponential midpoint, dt = 100 Delta t_CFL."""
    g = Grid(nx, nx, BC_DIRICHLET0)
    X, Y = cell_centres(g)
    bx, by, w = b_stream(X, Y, seed)
    dperp = 10.0 ** np.random.default_rng(seed + 1).uniform(-6.0, -2.0)
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, 1.0, dperp, w)
    pos = np.random.default_rng(seed + 2).uniform(-0.9, 0.9, size=(16, 2))
    gsrc = np.zeros_like(X)
    for xc, yc in pos:
        gsrc += gaussian(X, Y, xc, yc, 0.02)
    cfl = cfl_dt(g, Dxx, Dxy, Dyy)
    return Problem(f"c2-{nx}sq-dirichlet-stream-midpoint", g, Dxx, Dxy, Dyy,
                   source=SeparableSource([gsrc], [lambda t: 1.0]),
                   u0=gaussian(X, Y, 0.0, 0.0, 0.2), dt=100.0 * cfl, steps=steps, s=1,
                   c=(0.5,), tol=tol, cfl=cfl)


def config3_slices(nslices: int = 128, seed: int = 3, sides=(256, 512, 1024, 2048)):
    """Momentum-slice batch: per slice a side drawn uniformly from ``sides``
    (seed 3), p_s log-spaced in [1, 1e4] GeV, D_par = p^0.5, D_perp = 1e-3 D_par,
    shared circular b, a = (0.05, 0), constant Gaussian source (amp 1, sigma 0.1,
    origin), Gaussian u0 (sigma 0.2).  Returns (list of (side, D_par, D_perp))."""
    rng = np.random.default_rng(seed)
    side = rng.choice(np.asarray(sides), size=nslices)
    p = np.logspace(0.0, 4.0, nslices)
    dpar = np.sqrt(p)
    return [(int(side[s]), float(dpar[s]), float(1e-3 * dpar[s])) for s in range(nslices)]


def slice_problem(side: int, dpar: float, dperp: float, dt: float, tol: float = 1e-6,
                  steps: int = 10) -> Problem:
    g = Grid(side, side, BC_DIRICHLET0)
    X, Y = cell_centres(g)
    bx, by, w = b_circular(X, Y, 0.05)
    Dxx, Dxy, Dyy = tensor_from_b(bx, by, dpar, dperp, w)
    cfl = cfl_dt(g, Dxx, Dxy, Dyy)
    return Problem(f"slice-{side}-dpar{dpar:.3g}", g, Dxx, Dxy, Dyy, ax=0.05, ay=0.0,
                   source=SeparableSource([gaussian(X, Y, 0.0, 0.0, 0.1)], [lambda t: 1.0]),
                   u0=gaussian(X, Y, 0.0, 0.0, 0.2), dt=dt, steps=steps, s=1, c=(0.5,),
                   tol=tol, cfl=cfl)


def small_problem(nx: int, ny: int, bc: int, kind: str = "stream", seed: int = 7,
                  adv=(0.0, 0.0), adv_field: bool = False, dt_factor: float = 50.0,
                  s: int = 1, c=(0.5,), tol: float = 1e-10, tds: bool = False) -> Problem:
    """Small seeded cases for parity tests (ragged sizes allowed)."""
    g = Grid(nx, ny, bc)
    X, Y = cell_centres(g)
    if kind == "uniform":
        bx, by = b_uniform(X.shape, 30.0)
        Dxx, Dxy, Dyy = tensor_from_b(bx, by, 1.0, 1e-3)
    elif kind == "circular":
        bx, by, w = b_circular(X, Y, 0.05)
        Dxx, Dxy, Dyy = tensor_from_b(bx, by, 1.0, 1e-4, w)
    elif kind == "stream":
        bx, by, w = b_stream(X, Y, seed)
        Dxx, Dxy, Dyy = tensor_from_b(bx, by, 1.0, 1e-3, w)
    elif kind == "random":
        rng = np.random.default_rng(seed)
        # symmetric positive definite random tensor per cell
        l1 = rng.uniform(0.1, 1.0, X.shape)
        l2 = rng.uniform(0.001, 0.1, X.shape)
        th = rng.uniform(0, np.pi, X.shape)
        bx, by = np.cos(th), np.sin(th)
        Dxx = l2 + (l1 - l2) * bx * bx
        Dyy = l2 + (l1 - l2) * by * by
        Dxy = (l1 - l2) * bx * by
    else:
        from .fields import D_ring, D_spiral1, D_spiral2
        Dxx, Dxy, Dyy = {"ring": D_ring, "spiral1": D_spiral1, "spiral2": D_spiral2}[kind](X, Y)
    rng = np.random.default_rng(seed + 100)
    axf = ayf = None
    if adv_field:
        axf = adv[0] * (1.0 + 0.5 * np.sin(np.pi * X) * np.cos(np.pi * Y))
        ayf = adv[1] * (1.0 + 0.5 * np.cos(np.pi * X + 0.3))
    if tds:
        from .fields import tds_source
        src = tds_source(X, Y)
    else:
        src = SeparableSource([gaussian(X, Y, 0.1, -0.2, 0.15), rng.uniform(0, 0.1, X.shape)],
                              [lambda t: 1.0 + 0.5 * float(np.sin(2 * np.pi * t)), lambda t: 1.0])
    cfl = cfl_dt(g, Dxx, Dxy, Dyy)
    u0 = gaussian(X, Y, 0.0, 0.1, 0.25) + 0.01 * rng.standard_normal(X.shape)
    return Problem(f"small-{nx}x{ny}-{kind}-bc{bc}", g, Dxx, Dxy, Dyy, ax=adv[0], ay=adv[1],
                   ax_field=axf, ay_field=ayf, source=src, u0=u0, dt=dt_factor * cfl,
                   steps=1, s=s, c=tuple(c), tol=tol, cfl=cfl)


def paper_case(case: str, nx: int = 128) -> Problem:
    """The paper's own test problems (Section 3) on [-1,1]^2, zero Dirichlet.

    case "I":   diffusion along rings (Eq. B_ring), no advection, no source, T = 0.75
    case "II":  spiral 2 (Eq. B_spiral), a = (1, 1), time-independent sources (Eq. TIS), T = 0.85
    case "III": spiral 1 (Eq. B_spiral), a = (1, 1), time-dependent sources (Eq. TDS), T = 0.10
    case "IV":  spiral 2 (Eq. B_spiral), a = (1, 2), time-dependent sources (Eq. TDS), T = 0.10

    The paper gives neither the grid, the boundary condition nor the initial
    field; the readings are an nx^2 grid, zero Dirichlet, and a Gaussian of
    sigma 0.1 centred on the field lines at (0, 0.6).  ``dt`` holds the final
    time T and ``cfl`` the explicit step bound.
    """
    from .fields import D_ring, D_spiral1, D_spiral2, tds_source, tis_source
    g = Grid(nx, nx, BC_DIRICHLET0)
    X, Y = cell_centres(g)
    if case == "I":
        Dxx, Dxy, Dyy = D_ring(X, Y)
        ax, ay, src, T = 0.0, 0.0, SeparableSource(), 0.75
    elif case == "II":
        Dxx, Dxy, Dyy = D_spiral2(X, Y)
        ax, ay, src, T = 1.0, 1.0, tis_source(X, Y), 0.85
    elif case == "III":
        Dxx, Dxy, Dyy = D_spiral1(X, Y)
        ax, ay, src, T = 1.0, 1.0, tds_source(X, Y), 0.10
    elif case == "IV":
        Dxx, Dxy, Dyy = D_spiral2(X, Y)
        ax, ay, src, T = 1.0, 2.0, tds_source(X, Y), 0.10
    else:
        raise ValueError(f"unknown case {case!r}")
    u0 = gaussian(X, Y, 0.0, 0.6, 0.1)
    return Problem(f"paper-{case}-{nx}sq", g, Dxx, Dxy, Dyy, ax=ax, ay=ay, source=src, u0=u0,
                   dt=T, steps=1, cfl=cfl_dt(g, Dxx, Dxy, Dyy))
