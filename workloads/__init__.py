"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package holds no arithmetic of the DG method: it only builds meshes
(vertex coordinates and face connectivity), names the physical parameters of
each workload, and draws seeded random vectors.  Both the CPU oracle and the
CUDA path consume what it produces; neither imports the other.
"""
from .mesh import Mesh, box_mesh, clustered_spacing, mapped_box_mesh, ogrid_mesh  # noqa: F401
from .configs import (  # noqa: F401
    Physics, BC_PERIODIC, BC_DIRICHLET, BC_ISO_WALL, BC_ADIA_WALL, BC_FARFIELD,
    FIELD_UNIFORM, FIELD_VORTEX, FIELD_POISEUILLE, FIELD_TGV, FIELD_CYLINDER, FIELD_SHOCK,
    RIEMANN_ROE, RIEMANN_HLLC, RIEMANN_HLL, RIEMANN_LF, RIEMANN_AUSM, FORCING_NONE, FORCING_POISEUILLE,
    vortex_case, poiseuille_case, tgv_case, tgv_dt, cylinder_case, small_tgv_case,
    wavy_box_case, rotated_box_case, rotation_matrix, small_cylinder_case, swbli_case,
    wall_spacing,
)
from .random import random_direction, perturbation, mlp_params  # noqa: F401
