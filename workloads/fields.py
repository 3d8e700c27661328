"""Coefficient fields, sources and initial data on a cell-centred grid.

Conventions (shared by every consumer):
  * the domain is [x0, x1] x [y0, y1], split into nx x ny cells;
  * arrays are row-major ``[ny][nx]`` (x fastest), float64;
  * cell centres are x_i = x0 + (i + 1/2) dx, y_j = y0 + (j + 1/2) dy.

The diffusion tensor is D = [[D_xx, D_xy], [D_xy, D_yy]] (Section 1, the
tensor below Eq. anidiff; symmetric, D_yx = D_xy).  Field-aligned tensors are
built as D = D_perp I + (D_par - D_perp) b b^T for a unit vector field b.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Sequence

import numpy as np

BC_PERIODIC = 0
BC_DIRICHLET0 = 1


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    bc: int = BC_PERIODIC
    x0: float = -1.0
    x1: float = 1.0
    y0: float = -1.0
    y1: float = 1.0

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny

    @property
    def n(self) -> int:
        return self.nx * self.ny


def cell_centres(g: Grid):
    """Return (X, Y), each ``[ny][nx]`` float64, at the cell centres."""
    x = g.x0 + (np.arange(g.nx) + 0.5) * g.dx
    y = g.y0 + (np.arange(g.ny) + 0.5) * g.dy
    X, Y = np.meshgrid(x, y, indexing="xy")
    return X, Y


def tensor_from_b(bx, by, dpar, dperp, iso_weight=None):
    """D = D_perp I + (D_par - D_perp) M with M = w b b^T + (1 - w) I / 2.

    ``iso_weight`` is w (1 = purely field aligned); None means w = 1.
    Returns (Dxx, Dxy, Dyy) as float64 arrays broadcast to bx's shape.
    """
    bx = np.asarray(bx, dtype=np.float64)
    by = np.asarray(by, dtype=np.float64)
    w = np.ones_like(bx) if iso_weight is None else np.asarray(iso_weight, dtype=np.float64)
    mxx = w * bx * bx + (1.0 - w) * 0.5
    myy = w * by * by + (1.0 - w) * 0.5
    mxy = w * bx * by
    dd = dpar - dperp
    return dperp + dd * mxx, dd * mxy, dperp + dd * myy


def b_uniform(shape, angle_deg: float):
    a = np.deg2rad(angle_deg)
    return np.full(shape, np.cos(a)), np.full(shape, np.sin(a))


def b_circular(X, Y, r_smooth: float = 0.05):
    """Circular field lines b = (-y, x)/r, blended to isotropic for r < r_smooth.

    Returns (bx, by, w) with w = min(1, (r / r_smooth)^2) the field-aligned weight.
    """
    r = np.hypot(X, Y)
    safe = np.where(r > 0, r, 1.0)
    bx = np.where(r > 0, -Y / safe, 1.0)
    by = np.where(r > 0, X / safe, 0.0)
    w = np.minimum(1.0, (r / r_smooth) ** 2)
    return bx, by, w


def b_stream(X, Y, seed: int, nmodes: int = 8, smooth_frac: float = 0.05):
    """Field lines of a random-phase stream function.

    psi = sum_k A_k sin(pi (m_k x + n_k y) + phi_k), integer m_k, n_k in 1..4,
    A_k ~ U(0.5, 1), phi_k ~ U(0, 2 pi), all drawn from ``seed``.
    b = (d psi/dy, -d psi/dx) / |grad psi|, blended to isotropic where
    |grad psi| < smooth_frac * max |grad psi| with weight (|grad psi| / thr)^2.
    """
    rng = np.random.default_rng(seed)
    m = rng.integers(1, 5, size=nmodes)
    n = rng.integers(1, 5, size=nmodes)
    amp = rng.uniform(0.5, 1.0, size=nmodes)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=nmodes)
    px = np.zeros_like(X)
    py = np.zeros_like(X)
    for k in range(nmodes):
        c = amp[k] * np.pi * np.cos(np.pi * (m[k] * X + n[k] * Y) + ph[k])
        px += m[k] * c
        py += n[k] * c
    g = np.hypot(px, py)
    thr = smooth_frac * float(g.max())
    safe = np.where(g > 0, g, 1.0)
    bx = np.where(g > 0, py / safe, 1.0)
    by = np.where(g > 0, -px / safe, 0.0)
    w = np.minimum(1.0, (g / thr) ** 2) if thr > 0 else np.ones_like(g)
    return bx, by, w


# Paper's analytic tensors (Section 3): rank-one, no perpendicular diffusion.
def D_ring(X, Y):
    """Eq. B_ring: D_R = [[y^2, -xy], [-xy, x^2]]."""
    return Y * Y, -X * Y, X * X


def D_spiral1(X, Y):
    """Eq. B_spiral, first tensor: [[(x+y)^2, -x^2-xy], [-x^2-xy, x^2]]."""
    return (X + Y) ** 2, -X * X - X * Y, X * X


def D_spiral2(X, Y):
    """Eq. B_spiral, second tensor: [[(x+4y)^2, -x^2-4xy], [-x^2-4xy, x^2]]."""
    return (X + 4 * Y) ** 2, -X * X - 4 * X * Y, X * X


def gaussian(X, Y, xc, yc, sigma, amp=1.0):
    """amp * exp(-((x-xc)^2 + (y-yc)^2) / (2 sigma^2))."""
    return amp * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2.0 * sigma * sigma))


def gaussian_w(X, Y, xc, yc, w, amp=1.0):
    """The paper's form amp * exp(-((x-xc)^2 + (y-yc)^2) / w) (Eqs. TIS, TDS)."""
    return amp * np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / w)


@dataclass
class SeparableSource:
    """S(x, y, t) = sum_k h_k(t) g_k(x, y): spatial fields and time profiles."""
    g: List[np.ndarray] = field(default_factory=list)
    h: List[Callable[[float], float]] = field(default_factory=list)

    def coeffs(self, t: float) -> np.ndarray:
        return np.array([float(hk(t)) for hk in self.h], dtype=np.float64)

    def __len__(self):
        return len(self.g)


def _const(v):
    return lambda t: v


def tis_source(X, Y) -> SeparableSource:
    """Eq. TIS: 0.1 + 30 exp(-r_1^2 / 2.5e-2) + 40 exp(-r_2^2 / 3e-2)."""
    g = (np.full_like(X, 0.1)
         + gaussian_w(X, Y, -0.6, 0.75, 2.5e-2, 30.0)
         + gaussian_w(X, Y, 0.75, -0.8, 3e-2, 40.0))
    return SeparableSource([g], [_const(1.0)])


def tds_source(X, Y) -> SeparableSource:
    """Eq. TDS: three Gaussians, each times exp(-k |t - t0|)."""
    spec = [(100.0, 0.25, 0.25, 1.5e-2, 10.0, 0.1),
            (70.0, 0.4, -0.4, 2.5e-2, 5.0, 0.3),
            (50.0, -0.6, 0.6, 1.5e-2, 7.5, 0.6)]
    g, h = [], []
    for amp, xc, yc, w, k, t0 in spec:
        g.append(gaussian_w(X, Y, xc, yc, w, amp))
        h.append(lambda t, k=k, t0=t0: float(np.exp(-k * abs(t - t0))))
    return SeparableSource(g, h)


def cfl_dt(g: Grid, Dxx, Dxy, Dyy) -> float:
    """Explicit-Euler limit dx^2 / (4 max lambda_max(D)) used to size time steps.

    The paper quotes step sizes in multiples of Delta t_CFL without defining it;
    this is the isotropic 2-D forward-Euler bound with h = min(dx, dy).
    """
    tr = 0.5 * (Dxx + Dyy)
    disc = np.sqrt(0.25 * (Dxx - Dyy) ** 2 + Dxy ** 2)
    lmax = float(np.max(tr + disc))
    h = min(g.dx, g.dy)
    return h * h / (4.0 * lmax)
