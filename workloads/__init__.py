"""Seeded synthetic inputs for the anisotropic diffusion-advection problem.

This package only *generates inputs*: grids, cell-centred coefficient fields
D_xx, D_xy, D_yy and a_x, a_y, source terms g_k(x, y) with their time profiles
h_k(t), initial conditions and the workload descriptions.  It holds none of the
method's arithmetic (no discretisation, no Leja interpolation, no time
stepping), so both the CUDA path and the CPU oracle may import it.
"""
from .fields import (  # noqa: F401
    Grid, cell_centres, tensor_from_b, b_uniform, b_circular, b_stream,
    D_ring, D_spiral1, D_spiral2, gaussian, gaussian_w, SeparableSource,
    tis_source, tds_source, cfl_dt,
)
from .configs import (  # noqa: F401
    Problem, config0, config1, config2, config3_slices, slice_problem, small_problem,
)
