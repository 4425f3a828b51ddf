"""Seeded synthetic inputs for the acoustic DG wave solver.

This package builds the *inputs* of a solve -- hexahedral cube meshes (with
optional curving and relabelled element axes), coefficient fields, initial
states and the analytic solutions used to measure accuracy.  It holds none of the
discontinuous Galerkin arithmetic: no quadrature, no operator, no time
stepping.  Both the FP64 CPU oracle (``oracle/``) and the CUDA path
(``paper_1805_03981_gb300``) read what it produces, and it imports neither.
"""
from .mesh import cube_mesh, solution_node_positions, gll_points_1d  # noqa: F401
from . import fields, configs  # noqa: F401
