"""Hand-made mesh sets for the voxel tests (CPU and GPU)."""
import numpy as np


def empty_and_two_triangles():
    """Two objects over 2 LoDs: object 0 without facets, object 1 two
    parallel triangles one unit apart."""
    from synth.mesh import MeshSet
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1]], np.float32)
    V = np.ascontiguousarray(tri)
    F = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    vo = np.array([0, 0, 6], np.int64)
    fo = np.array([0, 0, 2], np.int64)
    z = np.zeros(2, np.float32)
    return MeshSet(n=2, n_lods=2, verts=[V, V], vert_off=[vo, vo], faces=[F, F], face_off=[fo, fo],
                   hd=[z, None], ph=[z.copy(), None], anchor=np.array([[0, 0, 0], [0, 0, 0]], np.float32),
                   kind="explicit")
