"""Seeded synthetic workload generators (meshes, materials, sources).

This package is shared input plumbing: it builds the arrays that both the
FP64 oracle and the GPU library receive (cells, faces, unit normals, areas,
volumes, cross sections, sources).  It holds none of the sweep method's
arithmetic: no direction sets, no upwind classification, no DAG, no solve.
"""

from .meshes import hex_grid, kuhn_tets, column_mesh, pinwheel_mesh  # noqa: F401
from .workloads import (  # noqa: F401
    WORKLOADS,
    make_workload,
    lognormal_blocks_sigma,
    batch_problem_specs,
    make_batch_problem,
    multigroup_materials,
    tets_edge_for_cells,
    QUAD_BY_NDIRS,
)
