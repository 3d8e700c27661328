"""Pins of the oracle's spectral bounds (Section 2: Gershgorin estimate of the
largest-magnitude eigenvalue, smallest taken as 0) and of the counter-based
generator used for the power-iteration start vector."""
import numpy as np
import pytest

from oracle import operator as op
from oracle import spectral
from workloads import Grid, config0, small_problem
from workloads.fields import BC_DIRICHLET0, BC_PERIODIC


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_DIRICHLET0])
@pytest.mark.parametrize("kind", ["random", "circular", "ring"])
def test_gershgorin_bounds_every_eigenvalue(bc, kind):
    p = small_problem(10, 12, bc, kind, adv=(0.6, -0.3), adv_field=True)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy, p.ax_arr(), p.ay_arr())
    alpha = spectral.gershgorin(A)
    ev = np.linalg.eigvals(A.toarray())
    assert alpha <= ev.real.min() + 1e-9 * abs(alpha)
    # disc radius from the dense rows, written out independently
    D = A.toarray()
    bound = min(D[i, i] - (np.abs(D[i]).sum() - abs(D[i, i])) for i in range(D.shape[0]))
    assert abs(bound - alpha) <= 1e-12 * abs(alpha)


def test_gershgorin_c0_closed_form():
    # constant coefficients: the diagonal is -2 (Dxx/dx^2 + Dyy/dy^2); the
    # off-diagonal magnitudes are Dxx/dx^2 (x2), Dyy/dy^2 (x2) and
    # |Dxy|/(2 dx dy) (x4 corners); the mixed contributions to E/W/N/S cancel.
    p = config0()
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy)
    Dxx, Dxy, Dyy = p.Dxx[0, 0], p.Dxy[0, 0], p.Dyy[0, 0]
    dx, dy = p.grid.dx, p.grid.dy
    expect = -4 * (Dxx / dx ** 2 + Dyy / dy ** 2) - 2 * abs(Dxy) / (dx * dy)
    assert abs(spectral.gershgorin(A) - expect) <= 1e-12 * abs(expect)
    assert abs(expect - (-4986.0192)) < 1e-3


def test_power_iteration_symmetric_extreme_eigenvalue():
    # a = 0 and D_xy = 0 give a symmetric A: compare with LAPACK's eigvalsh.
    g = Grid(12, 12, BC_DIRICHLET0)
    rng = np.random.default_rng(5)
    Dxx = rng.uniform(0.5, 1.5, (12, 12))
    Dyy = rng.uniform(0.1, 0.4, (12, 12))
    A = op.assemble(g, Dxx, 0.0, Dyy)
    assert abs(A - A.T).max() < 1e-10
    lam = np.linalg.eigvalsh(A.toarray())
    x0 = spectral.splitmix64_uniform(g.n, 11)
    alpha, est = spectral.power_iteration(A, x0, iters=3000, safety=1.1)
    assert abs(est - abs(lam).max()) <= 1e-6 * abs(lam).max()
    assert abs(alpha - (-1.1 * est)) < 1e-12 * abs(alpha)


def test_power_iteration_c0_converges_to_symbol_minimum():
    p = config0(nx=16)
    A = op.assemble(p.grid, p.Dxx, p.Dxy, p.Dyy)
    Dsum = p.Dxx[0, 0] + p.Dyy[0, 0]
    expect = 4 * Dsum / p.grid.dx ** 2          # theta = (pi, pi) of the symbol
    _, est = spectral.power_iteration(A, spectral.splitmix64_uniform(p.grid.n, 1), iters=4000)
    assert abs(est - expect) <= 1e-6 * expect


def test_splitmix64_published_outputs_and_counter_form():
    # SplitMix64 seeded with 0: first outputs 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4.
    M = (1 << 64) - 1
    state = 0
    seq = []
    for _ in range(3):                  # the sequential reference form
        state = (state + 0x9E3779B97F4A7C15) & M
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        seq.append(z ^ (z >> 31))
    assert seq[0] == 0xE220A8397B1DCDAF and seq[1] == 0x6E789E6AA1B965F4
    u = spectral.splitmix64_uniform(3, 0)
    assert np.array_equal(u, np.array([(s >> 11) * 2.0 ** -53 - 0.5 for s in seq]))
    big = spectral.splitmix64_uniform(20000, 42)
    assert -0.5 <= big.min() and big.max() < 0.5 and abs(big.mean()) < 0.01
