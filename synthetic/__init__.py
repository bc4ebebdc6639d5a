"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package generates mesh arrays (vertices, cells, Dirichlet vertex flags)
and random right-hand sides.  It holds none of the multigrid method's
arithmetic: no basis functions, quadrature, DoF numbering, operators or
transfers.  Both the oracle and the GPU library consume its output as input.
"""
from .meshes import (  # noqa: F401
    Level, splitmix64, uniform_pm1, structured_grid, jitter_interior,
    deform_sine, config_levels, CONFIGS,
)
from .rhs import normal_rhs  # noqa: F401
