"""Plain FP64 CPU oracle for the exponential Leja integrators of
Deka, Kissmann & Einkemmer (ICRC 2023), "Efficient numerical methods for
Anisotropic Diffusion of Galactic Cosmic Rays".

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute anything in this package: only the test-suite, the smoke check of the
package entry point and the CPU-baseline leg of the benchmark use it.  It
shares no code with the CUDA path (no kernels, headers, helpers, tables or
constant generators); the only common dependency is the seeded input
generator package ``workloads``, which holds none of the method's arithmetic.

Every function cites the passage of the paper it follows.  Modules:
  operator    -- sparse (CSR) assembly of A = div(D grad .) + div(a .)   (Eq. anidiff)
  spectral    -- Gershgorin and power-iteration bounds of the spectrum   (Section 2)
  leja        -- Leja points, divided differences, Newton recurrence,
                 phi_1 and augmented-matrix exponential                 (Section 2)
  integrators -- exponential midpoint, s-stage exponential quadrature   (Eqs. exp_quad,
                 exp_midpoint, exp_quad_Gauss)
  cn          -- Crank-Nicolson with an own restarted GMRES             (Section 3, comparison)
  mlp         -- NumPy reference of the spectral-bound predictor network

Parity status: every function here is pinned by a CPU test against closed
forms, invariants or brute force (tests/test_oracle_*.py); see the module
docstrings for the pins.
"""
