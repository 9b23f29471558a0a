"""Host-side input helpers of bench.py (CPU): the box candidates fed to the
voxel-pair filter record equal a brute-force box test, and the per-object
boxes equal the vertices' extremes."""
import numpy as np

import bench
from synth import configs


def test_object_boxes_are_vertex_extremes():
    S = configs.blob_set(50, 40.0, 3, 1)
    b = bench._object_boxes(S)
    for o in (0, 17, 49):
        v = S.object_verts(S.n_lods - 1, o)
        assert np.array_equal(b[o, :3], v.min(0)) and np.array_equal(b[o, 3:], v.max(0))


def test_box_candidates_equal_brute_force():
    R = configs.tube_set(25, 300.0, 1, 0, length_range=(50.0, 300.0))
    S = configs.blob_set(2500, 300.0, 1, 1)
    for tau in (0.0, 2.0, 15.0):
        pr, ps = bench.box_candidates(R, S, tau)
        a, b = bench._object_boxes(R), bench._object_boxes(S)
        g = np.maximum(0.0, np.maximum(b[None, :, :3] - a[:, None, 3:], a[:, None, :3] - b[None, :, 3:]))
        r, s = np.nonzero((g * g).sum(2) <= tau * tau)
        assert np.array_equal(pr, r) and np.array_equal(ps, s)
        assert len(pr) > 0

