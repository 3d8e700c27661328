"""Sparse assembly of the spatial operator A of Eq. anidiff (oracle).

Eq. anidiff (Section 1) reads du/dt = div(D grad u) + div(a u) + S, and the
paper writes A = div(D grad(.)) + div(a .) (Section 2, below Eq. exp_quad).
The paper does not give its spatial discretisation; the reading used here is a
conservative flux form on a cell-centred grid (a 9-point stencil):

  Fx(i+1/2, j) = Dxx_e (u(i+1,j) - u(i,j)) / dx
               + Dxy_e (u(i+1,j+1) + u(i,j+1) - u(i+1,j-1) - u(i,j-1)) / (4 dy)
               + ax_e (u(i,j) + u(i+1,j)) / 2
  Fy(i, j+1/2) = Dyy_n (u(i,j+1) - u(i,j)) / dy
               + Dxy_n (u(i+1,j+1) + u(i+1,j) - u(i-1,j+1) - u(i-1,j)) / (4 dx)
               + ay_n (u(i,j) + u(i,j+1)) / 2
  (A u)(i,j)   = (Fx(i+1/2,j) - Fx(i-1/2,j)) / dx + (Fy(i,j+1/2) - Fy(i,j-1/2)) / dy

Face coefficients are the mean of the two adjacent cells.  Boundaries:
  periodic   -- indices wrap (corners included);
  dirichlet0 -- ghost cells by odd reflection, u(-1, j) = -u(0, j), and a
                corner ghost is the diagonal mirror with sign +; ghost
                *coefficients* mirror without sign, so a boundary face takes
                the adjacent cell's value.  The cross-derivative and advective
                fluxes through a boundary face then vanish.

Two independent formulations live here: ``assemble`` builds the CSR matrix
term by term; ``apply_padded`` evaluates the flux formula on a ghost-padded
array without any matrix.  The tests pin both against each other, against the
continuous operator (second-order convergence) and against the exact Fourier
symbol for constant coefficients.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

BC_PERIODIC = 0
BC_DIRICHLET0 = 1


def _ghost_map(i, j, nx, ny, bc):
    """Map (possibly ghost) cell indices in [-1, n] to (interior flat index, sign)."""
    i = np.asarray(i)
    j = np.asarray(j)
    if bc == BC_PERIODIC:
        return (j % ny) * nx + (i % nx), np.ones(np.broadcast(i, j).shape)
    sign = np.ones(np.broadcast(i, j).shape)
    ii = np.where(i < 0, -1 - i, np.where(i >= nx, 2 * nx - 1 - i, i))
    jj = np.where(j < 0, -1 - j, np.where(j >= ny, 2 * ny - 1 - j, j))
    sign = sign * np.where((i < 0) | (i >= nx), -1.0, 1.0)
    sign = sign * np.where((j < 0) | (j >= ny), -1.0, 1.0)
    return jj * nx + ii, sign


def _coef(field, i, j, nx, ny, bc):
    """Coefficient value at a (possibly ghost) cell: mirrored/wrapped, no sign."""
    idx, _ = _ghost_map(i, j, nx, ny, bc)
    return field.reshape(-1)[idx]


def _east_face_terms(I, J, F, dx, dy, nx, ny, bc):
    """Terms (coef, di, dj) of Fx at the east face of cells (I, J) (I may be -1)."""
    Dxx, Dxy, Dyy, ax, ay = F
    cxx = 0.5 * (_coef(Dxx, I, J, nx, ny, bc) + _coef(Dxx, I + 1, J, nx, ny, bc))
    cxy = 0.5 * (_coef(Dxy, I, J, nx, ny, bc) + _coef(Dxy, I + 1, J, nx, ny, bc))
    cax = 0.5 * (_coef(ax, I, J, nx, ny, bc) + _coef(ax, I + 1, J, nx, ny, bc))
    q = cxy / (4.0 * dy)
    return [(cxx / dx, 1, 0), (-cxx / dx, 0, 0),
            (q, 1, 1), (q, 0, 1), (-q, 1, -1), (-q, 0, -1),
            (0.5 * cax, 0, 0), (0.5 * cax, 1, 0)]


def _north_face_terms(I, J, F, dx, dy, nx, ny, bc):
    """Terms (coef, di, dj) of Fy at the north face of cells (I, J) (J may be -1)."""
    Dxx, Dxy, Dyy, ax, ay = F
    cyy = 0.5 * (_coef(Dyy, I, J, nx, ny, bc) + _coef(Dyy, I, J + 1, nx, ny, bc))
    cxy = 0.5 * (_coef(Dxy, I, J, nx, ny, bc) + _coef(Dxy, I, J + 1, nx, ny, bc))
    cay = 0.5 * (_coef(ay, I, J, nx, ny, bc) + _coef(ay, I, J + 1, nx, ny, bc))
    q = cxy / (4.0 * dx)
    return [(cyy / dy, 0, 1), (-cyy / dy, 0, 0),
            (q, 1, 1), (q, 1, 0), (-q, -1, 1), (-q, -1, 0),
            (0.5 * cay, 0, 0), (0.5 * cay, 0, 1)]


def _fields(grid, Dxx, Dxy, Dyy, ax, ay):
    shape = (grid.ny, grid.nx)

    def as_field(v):
        a = np.asarray(v, dtype=np.float64)
        return np.broadcast_to(a, shape).astype(np.float64)
    return tuple(as_field(v) for v in (Dxx, Dxy, Dyy, ax, ay))


def assemble(grid, Dxx, Dxy, Dyy, ax=0.0, ay=0.0) -> sp.csr_matrix:
    """CSR matrix of A (Eq. anidiff, A as defined below Eq. exp_quad).

    ``ax``/``ay`` may be scalars (constant advection) or ``[ny][nx]`` fields.
    Duplicate entries (the same column reached through two ghosts or two
    faces) are summed, so the matrix holds the true entries a_ij.
    """
    nx, ny, bc = grid.nx, grid.ny, grid.bc
    dx, dy = grid.dx, grid.dy
    F = _fields(grid, Dxx, Dxy, Dyy, ax, ay)
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    I = I.reshape(-1)
    J = J.reshape(-1)
    rows = J * nx + I
    R, C, V = [], [], []

    def add(terms, I0, J0, scale):
        for coef, di, dj in terms:
            col, sgn = _ghost_map(I0 + di, J0 + dj, nx, ny, bc)
            R.append(rows)
            C.append(col)
            V.append(scale * sgn * np.broadcast_to(coef, rows.shape))

    add(_east_face_terms(I, J, F, dx, dy, nx, ny, bc), I, J, 1.0 / dx)
    add(_east_face_terms(I - 1, J, F, dx, dy, nx, ny, bc), I - 1, J, -1.0 / dx)
    add(_north_face_terms(I, J, F, dx, dy, nx, ny, bc), I, J, 1.0 / dy)
    add(_north_face_terms(I, J - 1, F, dx, dy, nx, ny, bc), I, J - 1, -1.0 / dy)
    A = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))),
                      shape=(grid.n, grid.n)).tocsr()
    A.sum_duplicates()
    A.eliminate_zeros()
    return A


def pad_ghost(u, bc, sign=True):
    """Return u padded by one ghost layer following the boundary rule.

    With ``sign=False`` the ghosts mirror without sign (used for coefficients).
    """
    u = np.asarray(u, dtype=np.float64)
    if bc == BC_PERIODIC:
        return np.pad(u, 1, mode="wrap")
    g = np.pad(u, 1, mode="symmetric")
    if sign:
        g[0, :] *= -1.0
        g[-1, :] *= -1.0
        g[:, 0] *= -1.0
        g[:, -1] *= -1.0
    return g


def apply_padded(grid, u, Dxx, Dxy, Dyy, ax=0.0, ay=0.0):
    """A u by direct evaluation of the face fluxes on ghost-padded arrays."""
    dx, dy, bc = grid.dx, grid.dy, grid.bc
    Dxx, Dxy, Dyy, ax, ay = _fields(grid, Dxx, Dxy, Dyy, ax, ay)
    U = pad_ghost(u, bc)
    cD = {k: pad_ghost(v, bc, sign=False) for k, v in
          dict(xx=Dxx, xy=Dxy, yy=Dyy, ax=ax, ay=ay).items()}
    ny, nx = u.shape
    # face fluxes Fx at x-faces k = 0..nx (between padded columns k and k+1)
    def P(arr, dj, di):  # view of padded array, rows 1+dj.., cols di..
        return arr[1 + dj:1 + dj + ny, di:di + nx + 1]
    avg = lambda a: 0.5 * (P(a, 0, 0) + P(a, 0, 1))
    Fx = (avg(cD["xx"]) * (P(U, 0, 1) - P(U, 0, 0)) / dx
          + avg(cD["xy"]) * (P(U, 1, 1) + P(U, 1, 0) - P(U, -1, 1) - P(U, -1, 0)) / (4 * dy)
          + avg(cD["ax"]) * (P(U, 0, 0) + P(U, 0, 1)) / 2)
    def Q(arr, dj, di):  # rows dj.., cols 1+di..
        return arr[dj:dj + ny + 1, 1 + di:1 + di + nx]
    avgy = lambda a: 0.5 * (Q(a, 0, 0) + Q(a, 1, 0))
    Fy = (avgy(cD["yy"]) * (Q(U, 1, 0) - Q(U, 0, 0)) / dy
          + avgy(cD["xy"]) * (Q(U, 1, 1) + Q(U, 0, 1) - Q(U, 1, -1) - Q(U, 0, -1)) / (4 * dx)
          + avgy(cD["ay"]) * (Q(U, 0, 0) + Q(U, 1, 0)) / 2)
    return (Fx[:, 1:] - Fx[:, :-1]) / dx + (Fy[1:, :] - Fy[:-1, :]) / dy


def fourier_symbol(grid, Dxx, Dxy, Dyy, ax, ay, thx, thy):
    """Exact eigenvalue of A on the mode exp(i (thx i + thy j)) for constant
    coefficients and periodic boundaries (derived from the flux form above)."""
    dx, dy = grid.dx, grid.dy
    return (-4.0 * Dxx / dx ** 2 * np.sin(thx / 2) ** 2
            - 4.0 * Dyy / dy ** 2 * np.sin(thy / 2) ** 2
            - 2.0 * Dxy / (dx * dy) * np.sin(thx) * np.sin(thy)
            + 1j * (ax * np.sin(thx) / dx + ay * np.sin(thy) / dy))
