"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds geometry and initial-state generators only: structured
meshes (face area vectors, volumes, centres, boundary tags), velocity-grid
descriptors and initial macroscopic fields.  It contains none of the method's
arithmetic (no moments, no reference distributions, no fluxes), so both the
oracle and the GPU path may import it without sharing any solver code.
"""
from .meshes import (  # noqa: F401
    BC_NONE, BC_FARFIELD, BC_WALL, BC_PERIODIC,
    Mesh, cartesian_1d, cartesian_2d, cylinder_ogrid, sphere_ogrid,
)
from .cases import (  # noqa: F401
    Case, VGrid, shock_1d_case, cylinder_case, sphere_case, shock_batch_cases,
    rankine_hugoniot, batch_vgrid_n, batch_vgrid_half_width,
)
