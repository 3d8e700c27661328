"""Pins the window argument of window_oracle.py: a cell of a forced-count
step computed on a window of radius k + 2 equals the full-grid oracle's
value (to rounding), and a window of radius k does not."""
import numpy as np
import pytest

from oracle import integrators
from oracle import operator as oop
from window_oracle import alpha_from_fields, oracle_cell, sample_cells
from workloads import config2, slice_problem


@pytest.mark.parametrize("k", [2, 7])
def test_window_cells_equal_full_grid_oracle(k):
    p = config2(nx=96)
    alpha = alpha_from_fields(p)
    g = p.source.g[0]
    A = oop.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, 0.0, 0.0)
    full, st = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,),
                                        lambda t: g.ravel(), alpha, tol=1e-10, force_iters=k)
    assert st.iters == k and st.substeps == 1
    full = full.reshape(p.grid.ny, p.grid.nx)
    pts = sample_cells(96, 96, 30, seed=3, strip=40)
    got = np.array([oracle_cell(p, i, j, k + 2, alpha, k, g) for i, j in pts])
    ref = np.array([full[j, i] for i, j in pts])
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    short = np.array([oracle_cell(p, i, j, k, alpha, k, g) for i, j in pts])
    assert np.abs(short - ref).max() > 1e-9 * np.abs(ref).max()


def test_window_cells_equal_full_grid_oracle_with_advection():
    """A batch slice: constant advection a = (0.05, 0) and a circular field."""
    k = 5
    p = slice_problem(64, 10.0, 1e-2, dt=1.0)
    p.dt = 100.0 * p.cfl
    alpha = alpha_from_fields(p)
    g = p.source.g[0]
    A = oop.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax, p.ay)
    full, _ = integrators.expquad_step(A, p.u0.ravel(), 0.0, p.dt, 1, (0.5,),
                                       lambda t: g.ravel(), alpha, tol=1e-10, force_iters=k)
    full = full.reshape(64, 64)
    pts = sample_cells(64, 64, 20, seed=5, strip=30)
    got = np.array([oracle_cell(p, i, j, k + 2, alpha, k, g) for i, j in pts])
    ref = np.array([full[j, i] for i, j in pts])
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
