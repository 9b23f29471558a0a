"""Seeded synthetic inputs: every object has its own counter-keyed random
stream, so a set generated in chunks (as the streamed workload and the
parallel generators do) is bit-identical to the set generated whole, and a
call with the same seed gives the same set.  Also the layout invariants the
loaders rely on: shared blob topology, hd / ph absent (zero) at the original
surface, non-negative elsewhere, offsets starting at 0 and non-decreasing,
anchors on the original surface."""
import numpy as np
import pytest

from synth import configs
from synth.mesh import concat


def same_set(a, b):
    assert a.n == b.n and a.n_lods == b.n_lods
    for f in ("verts", "vert_off", "faces", "face_off", "hd", "ph"):
        for x, y in zip(getattr(a, f), getattr(b, f)):
            assert (x is None) == (y is None), f
            if x is not None:
                assert np.array_equal(np.asarray(x), np.asarray(y)), f
    assert np.array_equal(a.anchor, b.anchor)


@pytest.mark.parametrize("cuts", [(0, 700, 1500), (0, 1, 1023, 1024, 1500), (0, 512, 1500)])
def test_blob_chunks_equal_whole(cuts):
    n, side = 1500, 60.0
    whole = configs.blob_set(n, side, 3, 0)
    parts = [configs.blob_set(n, side, 3, 0, start=a, count=b - a) for a, b in zip(cuts[:-1], cuts[1:])]
    same_set(concat(parts), whole)


def test_tube_chunks_equal_whole():
    n, side = 24, 200.0
    whole = configs.tube_set(n, side, 5, 1, length_range=(50.0, 90.0))
    parts = [configs.tube_set(n, side, 5, 1, start=a, count=b - a, length_range=(50.0, 90.0))
             for a, b in ((0, 7), (7, 8), (8, 24))]
    same_set(concat(parts), whole)


def test_stream_chunks_tile_the_set():
    n, chunks = 3000, 4
    whole = configs.blob_set(n, 5000.0, 0, 0)
    parts = [configs.stream2m_R_chunk(c, n=n, chunks=chunks) for c in range(chunks)]
    assert sum(p.n for p in parts) == n
    same_set(concat(parts), whole)


def test_seeds():
    a = configs.blob_set(200, 30.0, 7, 0)
    b = configs.blob_set(200, 30.0, 7, 0)
    c = configs.blob_set(200, 30.0, 8, 0)
    d = configs.blob_set(200, 30.0, 7, 1)
    same_set(a, b)
    assert not np.array_equal(a.verts[-1], c.verts[-1])
    assert not np.array_equal(a.verts[-1], d.verts[-1])


@pytest.mark.parametrize("kind", ["blob", "tube"])
def test_layout_invariants(kind):
    m = configs.blob_set(300, 40.0, 1, 0) if kind == "blob" else \
        configs.tube_set(10, 150.0, 1, 0, length_range=(50.0, 80.0))
    L = m.n_lods
    assert m.hd[L - 1] is None and m.ph[L - 1] is None
    for l in range(L):
        vo = np.asarray(m.vert_off[l])
        assert vo[0] == 0 and np.all(np.diff(vo) >= 0) and vo[-1] == m.verts[l].shape[0]
        if kind == "blob":
            assert m.face_off[l] is None   # one shared template per LoD
        else:
            fo = np.asarray(m.face_off[l])
            assert fo[0] == 0 and np.all(np.diff(fo) >= 0) and fo[-1] == m.faces[l].shape[0]
        for o in range(m.n):
            f = m.object_faces(l, o)
            assert f.min() >= 0 and f.max() < m.object_verts(l, o).shape[0]
        if l < L - 1:
            assert np.all(m.hd[l] >= 0) and np.all(m.ph[l] >= 0)
            assert m.hd[l].shape[0] == m.total_faces(l) == m.ph[l].shape[0]
        assert np.isfinite(m.verts[l]).all()
    # the anchor is a vertex of the original surface of its object
    for o in range(m.n):
        v = m.object_verts(L - 1, o)
        assert (np.abs(v - m.anchor[o]).max(axis=1) == 0).any()
