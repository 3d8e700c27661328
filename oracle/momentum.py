"""Momentum coupling of Eq. cr_full (oracle): the transport operator on (x, y, p).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU baseline, never by the product path.

Eq. cr_full (Section 1) adds to the spatial terms of Eq. anidiff the momentum
terms
    d/dp( p^2 D_pp d/dp(u / p^2) ) - d/dp( (pdot - (p/3) div v) u ) - (1/tau_f + 1/tau_r) u.
The paper integrates only the two-dimensional Eq. anidiff and names these
terms as future work (Sections 1 and 4).  Readings (each listed in the design
notes):
  * u(x, y, p) lives on the spatial grid of Eq. anidiff times np momentum
    cells with faces P_0 < P_1 < ... < P_np (any spacing; the workloads use
    logarithmic spacing), centres p_k = sqrt(P_k P_{k+1}) and widths
    dP_k = P_{k+1} - P_k;
  * the spatial diffusion tensor scales per momentum cell,
    D(x, y, p_k) = beta_k D(x, y); the advection a does not depend on p;
  * D_pp and b = pdot - (p/3) div v (div v constant in space) are given at the
    momentum faces, the loss rate L_k = 1/tau_f + 1/tau_r per cell;
  * finite volumes in p with no flux through P_0 and P_np:
        F_{k+1/2} = P_{k+1}^2 Dpp(P_{k+1}) (u_{k+1}/p_{k+1}^2 - u_k/p_k^2) / (p_{k+1} - p_k)
        G_{k+1/2} = b(P_{k+1}) * (u_k if b(P_{k+1}) >= 0 else u_{k+1})       (upwind)
        (A_p u)_k = (F_{k+1/2} - F_{k-1/2} - G_{k+1/2} + G_{k-1/2}) / dP_k - L_k u_k
  * unknowns are ordered slice-major: index k * n + (j * nx + i), so each
    momentum slice is one contiguous field of Eq. anidiff.

So A = blockdiag_k( A_xy(beta_k D, a) ) + kron(M, I_n), with A_xy the oracle
operator of Eq. anidiff (oracle.operator.assemble) and M the np x np momentum
matrix above.

Pins (tests/test_oracle_momentum.py): particle conservation (weighted column
sums vanish), the steady state u ~ p^2 of the momentum diffusion, the
Kronecker-sum structure of exp(tA) when beta = 1, second-order convergence of
the momentum diffusion against a symbolic derivative, the direction of the
upwind loss flux, and the exact decay of the loss term.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .operator import assemble


def centres(P):
    """Momentum cell centres p_k = sqrt(P_k P_{k+1}) and widths dP_k."""
    P = np.asarray(P, dtype=np.float64)
    return np.sqrt(P[:-1] * P[1:]), np.diff(P)


def momentum_matrix(P, dpp, b, loss) -> np.ndarray:
    """The np x np matrix M of the momentum terms (dense; np is small).

    P: np + 1 faces; dpp, b: np + 1 face values (the two boundary values are
    not used: no flux leaves the momentum range); loss: np cell rates."""
    P = np.asarray(P, dtype=np.float64)
    p, dP = centres(P)
    npm = len(p)
    if len(dpp) != npm + 1 or len(b) != npm + 1 or len(loss) != npm:
        raise ValueError("dpp and b need np + 1 face values, loss np cell values")
    M = np.zeros((npm, npm))
    for f in range(1, npm):            # interior face between cells f - 1 and f
        lo, hi = f - 1, f
        # diffusion flux F_f = K (u_hi / p_hi^2 - u_lo / p_lo^2)
        K = P[f] ** 2 * dpp[f] / (p[hi] - p[lo])
        flux = {hi: K / p[hi] ** 2, lo: -K / p[lo] ** 2}
        # upwind advective flux G_f = b_f u_up
        up = lo if b[f] >= 0 else hi
        adv = {up: b[f]}
        # the face adds +flux to the cell below it (as its upper face) and
        # -flux to the cell above (as its lower face); the advective flux the
        # other way round (-d/dp of b u)
        for col, v in flux.items():
            M[lo, col] += v / dP[lo]
            M[hi, col] -= v / dP[hi]
        for col, v in adv.items():
            M[lo, col] -= v / dP[lo]
            M[hi, col] += v / dP[hi]
    M -= np.diag(np.asarray(loss, dtype=np.float64))
    return M


def assemble3d(grid, Dxx, Dxy, Dyy, ax, ay, beta, M) -> sp.csr_matrix:
    """CSR matrix of the coupled operator, slice-major ordering."""
    n = grid.n
    blocks = [assemble(grid, bk * np.asarray(Dxx), bk * np.asarray(Dxy), bk * np.asarray(Dyy),
                       ax, ay) for bk in beta]
    A = sp.block_diag(blocks, format="csr") + sp.kron(sp.csr_matrix(M), sp.identity(n),
                                                      format="csr")
    return A.tocsr()
