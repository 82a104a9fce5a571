"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module draws random numbers and evaluates the coefficient fields that
define each workload.  It holds none of the method's arithmetic (no
assembly, no cyclic reduction, no H-matrix work): both implementations take
its arrays as plain inputs.

Grid convention (shared by every workload): ``n`` interior points per axis
on the unit cube, spacing ``h = 1/(n+1)``, node ``(ix, iy, iz)`` at
``((ix+1)h, (iy+1)h, (iz+1)h)``, flattened with x fastest:
``p = ix + n*iy + n*n*iz``.  Planes are the z-slices.
"""
from .fields import (  # noqa: F401
    grid_coords, gaussian_field_kappa, box_inclusions_kappa, codi_beta,
    uniform_rhs, workload, WORKLOADS, fd_cells, layered_speed, helmholtz_omega,
)
