"""Oracle values of single cells of a forced-count step on a large grid.

A step with a forced count of k Leja iterations changes a cell only through
the cells within k + 1 of it (one operator application for the right-hand
side, k in the series).  So the oracle computes a cell exactly on a window of
radius k + 2 around it: the window's own zero-Dirichlet edge is k + 2 cells
away from the cell, or is the domain's edge, where the window applies the
domain's rule.  tests/test_window_oracle.py pins this against the full-grid
oracle; the full-size GPU tests use it.  Test infrastructure only.
"""
import numpy as np

from oracle import integrators
from oracle import operator as oop
from workloads import Grid
from workloads.fields import BC_DIRICHLET0


def alpha_from_fields(p):
    """A spectral bound of the size of Gershgorin's, from the fields alone:
    -6 max lambda_max(D) (1/dx^2 + 1/dy^2)."""
    h = 0.5 * (p.Dxx - p.Dyy)
    lam = float(np.max(0.5 * (p.Dxx + p.Dyy) + np.sqrt(h * h + p.Dxy * p.Dxy)))
    return -6.0 * lam * (1.0 / p.grid.dx ** 2 + 1.0 / p.grid.dy ** 2)


def sample_cells(nx, ny, count, seed, strip=120):
    """Corners, edges, cells next to the FP32 kernels' strip and tile seams,
    and seeded interior cells."""
    pts = {(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1), (nx // 2, 0), (0, ny // 2),
           (nx - 1, ny // 2), (nx // 2, ny - 1), (1, 1), (2, ny - 3)}
    for x in (strip - 1, strip, 2 * strip - 1, 2 * strip, nx - strip, nx - 2):
        if 0 <= x < nx:
            pts.add((x, (x * 7) % ny))
    rng = np.random.default_rng(seed)
    while len(pts) < count:
        pts.add((int(rng.integers(0, nx)), int(rng.integers(0, ny))))
    return sorted(pts)


def oracle_cell(p, i, j, R, alpha, k, g_src):
    """u after one forced-count midpoint step at cell (i, j), from the window
    of radius R around it (zero-Dirichlet domain)."""
    g = p.grid
    assert g.bc == BC_DIRICHLET0
    i0, i1 = max(0, i - R), min(g.nx, i + R + 1)
    j0, j1 = max(0, j - R), min(g.ny, j + R + 1)
    wg = Grid(i1 - i0, j1 - j0, g.bc, x0=g.x0 + i0 * g.dx, x1=g.x0 + i1 * g.dx,
              y0=g.y0 + j0 * g.dy, y1=g.y0 + j1 * g.dy)
    sl = (slice(j0, j1), slice(i0, i1))
    A = oop.assemble(wg, p.Dxx[sl], p.Dxy[sl], p.Dyy[sl], float(p.ax), float(p.ay))
    gw = g_src[sl].ravel()
    S = lambda t: gw                      # time-independent sources (h = 1)
    u, _ = integrators.expquad_step(A, p.u0[sl].ravel(), 0.0, p.dt, 1, (0.5,), S, alpha,
                                    tol=1e-10, force_iters=k)
    return u.reshape(j1 - j0, i1 - i0)[j - j0, i - i0]
