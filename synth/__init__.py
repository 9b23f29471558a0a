"""Seeded synthetic inputs (meshes, LoDs, Hausdorff bounds) shared by the
CUDA path's tests and benchmark and by the CPU oracle's tests.  Holds none of
the join's arithmetic."""
from .mesh import MeshSet, icosphere, subdivision_map, real_sh_deg4, from_triangles, box_triangles, subset  # noqa: F401
from . import configs  # noqa: F401
