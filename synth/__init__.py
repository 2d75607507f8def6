"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package holds only input generation: mesh topology and vertex
coordinates, per-cell coefficient fields and the analytic functions that the
caller evaluates at quadrature points.  It contains none of the virtual
element arithmetic (no geometry moments, projections, matrices or solvers);
each side computes those itself.
"""

from .meshes import Mesh, hex_mesh, tet_mesh, prism_mesh, octa_mesh, affine, from_cell_loops, cell_vertex_ids  # noqa: F401
from . import fields  # noqa: F401
