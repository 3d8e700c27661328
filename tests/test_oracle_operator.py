"""Pins of the oracle's spatial operator (Eq. anidiff, A defined below Eq. exp_quad).

* two independent formulations (CSR term assembly vs. flux evaluation on
  ghost-padded arrays) agree on ragged grids, both boundary rules;
* constant coefficients + periodic: every Fourier mode is an eigenvector with
  the hand-derived symbol (diffusion, mixed term and advection, with signs);
* smooth fields: A u converges at second order to div(D grad u) + div(a u)
  (the sign of the advective term in Eq. anidiff is pinned here);
* conservation: 1^T A = 0 for periodic boundaries (any D, constant or field a).
"""
import numpy as np
import pytest

from oracle import operator as op
from workloads import Grid, small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_DIRICHLET0])
@pytest.mark.parametrize("nx,ny", [(5, 5), (7, 5), (17, 23), (3, 4)])
def test_csr_matches_padded_flux_form(bc, nx, ny):
    p = small_problem(nx, ny, bc, "random", adv=(0.7, -0.4), adv_field=True)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    u = np.random.default_rng(3).standard_normal((ny, nx))
    a1 = (A @ u.ravel()).reshape(ny, nx)
    a2 = op.apply_padded(p.grid, u, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    assert np.max(np.abs(a1 - a2)) <= 1e-14 * np.max(np.abs(a1))


def test_stencil_is_nine_point_and_dirichlet_folds():
    p = small_problem(6, 6, BC_PERIODIC, "random")
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy)
    assert A.getnnz(axis=1).max() == 9
    q = small_problem(6, 6, BC_DIRICHLET0, "random")
    B = op.assemble(q.grid, q.Dxx, q.Dxy, q.Dyy).toarray()
    # corner cell (0,0) couples only to (1,0), (0,1), (1,1) and itself
    assert set(np.nonzero(B[0])[0]) <= {0, 1, 6, 7}


@pytest.mark.parametrize("n", [8, 12])
def test_fourier_symbol_constant_coefficients(n):
    g = Grid(n, n + 2, BC_PERIODIC)
    Dxx, Dxy, Dyy, ax, ay = 0.8, 0.3, 0.25, 0.4, -0.7
    A = op.assemble(g, Dxx, Dxy, Dyy, ax, ay)
    I, J = np.meshgrid(np.arange(g.nx), np.arange(g.ny), indexing="xy")
    for kx in range(g.nx):
        for ky in range(g.ny):
            thx, thy = 2 * np.pi * kx / g.nx, 2 * np.pi * ky / g.ny
            mode = np.exp(1j * (thx * I + thy * J)).ravel()
            lam = op.fourier_symbol(g, Dxx, Dxy, Dyy, ax, ay, thx, thy)
            res = A @ mode.real + 1j * (A @ mode.imag)
            assert np.max(np.abs(res - lam * mode)) <= 1e-12 * max(1.0, abs(lam))


def test_c0_extreme_eigenvalue_closed_form():
    # 64^2, b at 30 deg, D_par 1, D_perp 1e-3: the symbol is most negative at
    # theta = (pi, pi): -4 (Dxx + Dyy) / dx^2 = -4 * 1.001 * 1024.
    from workloads import config0
    p = config0()
    Dxx, Dxy, Dyy = p.Dxx[0, 0], p.Dxy[0, 0], p.Dyy[0, 0]
    assert abs(Dxx - 0.75025) < 1e-12 and abs(Dyy - 0.25075) < 1e-12
    th = np.linspace(0, 2 * np.pi, 257)
    TX, TY = np.meshgrid(th, th)
    lam = op.fourier_symbol(p.grid, Dxx, Dxy, Dyy, 0.0, 0.0, TX, TY).real
    assert abs(lam.min() - (-4 * 1.001 * 1024)) < 1e-9


def _continuous_case():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    pi = sympy.pi
    u = sympy.sin(pi * x) * sympy.cos(pi * y) + sympy.Rational(1, 2) * sympy.sin(2 * pi * y + 0.3)
    Dxx = 1 + sympy.Rational(1, 2) * sympy.sin(pi * x) ** 2
    Dyy = sympy.Rational(3, 4) + sympy.Rational(1, 4) * sympy.cos(pi * y)
    Dxy = sympy.Rational(3, 10) * sympy.sin(pi * (x + y))
    ax = sympy.Rational(1, 2) + sympy.Rational(1, 4) * sympy.cos(pi * y)
    ay = -sympy.Rational(1, 3) + sympy.Rational(1, 5) * sympy.sin(pi * x)
    fx = Dxx * sympy.diff(u, x) + Dxy * sympy.diff(u, y) + ax * u
    fy = Dxy * sympy.diff(u, x) + Dyy * sympy.diff(u, y) + ay * u
    Au = sympy.diff(fx, x) + sympy.diff(fy, y)          # div(D grad u) + div(a u)
    lam = lambda e: sympy.lambdify((x, y), e, "numpy")
    return [lam(e) for e in (u, Dxx, Dxy, Dyy, ax, ay, Au)]


def test_second_order_consistency_periodic():
    fu, fDxx, fDxy, fDyy, fax, fay, fAu = _continuous_case()
    errs = []
    for n in (32, 64, 128):
        g = Grid(n, n, BC_PERIODIC)
        x = g.x0 + (np.arange(n) + 0.5) * g.dx
        X, Y = np.meshgrid(x, x)
        ev = lambda f: np.broadcast_to(f(X, Y), X.shape).astype(float)
        A = op.assemble(g, ev(fDxx), ev(fDxy), ev(fDyy), ev(fax), ev(fay))
        approx = (A @ ev(fu).ravel()).reshape(n, n)
        errs.append(np.max(np.abs(approx - ev(fAu))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


def test_second_order_consistency_dirichlet_interior():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    pi = sympy.pi
    u = sympy.sin(pi * (x + 1)) * sympy.sin(pi * (y + 1) / 2)     # vanishes on the boundary
    Dxx, Dyy, Dxy = 1 + x * x / 2, 1 - y / 4, sympy.Rational(1, 5) * (1 + x * y)
    ax, ay = sympy.Rational(3, 10), -sympy.Rational(1, 5)
    Au = (sympy.diff(Dxx * sympy.diff(u, x) + Dxy * sympy.diff(u, y) + ax * u, x)
          + sympy.diff(Dxy * sympy.diff(u, x) + Dyy * sympy.diff(u, y) + ay * u, y))
    f = [sympy.lambdify((x, y), e, "numpy") for e in (u, Dxx, Dxy, Dyy, Au)]
    errs = []
    for n in (32, 64, 128):
        g = Grid(n, n, BC_DIRICHLET0)
        c = g.x0 + (np.arange(n) + 0.5) * g.dx
        X, Y = np.meshgrid(c, c)
        ev = lambda h: np.broadcast_to(h(X, Y), X.shape).astype(float)
        A = op.assemble(g, ev(f[1]), ev(f[2]), ev(f[3]), 0.3, -0.2)
        r = (A @ ev(f[0]).ravel()).reshape(n, n) - ev(f[4])
        k = n // 8                                   # away from the boundary layer
        errs.append(np.max(np.abs(r[k:-k, k:-k])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


@pytest.mark.parametrize("adv_field", [False, True])
def test_periodic_column_sums_vanish(adv_field):
    p = small_problem(9, 11, BC_PERIODIC, "random", adv=(0.5, 0.2), adv_field=adv_field)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    colsum = np.asarray(A.sum(axis=0)).ravel()
    assert np.max(np.abs(colsum)) <= 1e-12 * abs(A).max()


def test_diffusion_annihilates_constants():
    for bc in (BC_PERIODIC,):
        p = small_problem(8, 8, bc, "random")
        A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy)
        assert np.max(np.abs(A @ np.ones(64))) <= 1e-12 * abs(A).max()
