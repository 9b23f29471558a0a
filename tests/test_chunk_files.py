"""Chunk files and the native chunk source (out-of-core streaming of R):
chunks written and read back bit for bit with every read-ahead depth, over
repeated passes and restarts, through the same fill entry point a streamed
join calls; the reader keeps to its buffer budget; damaged, truncated,
missing or changed files are reported.  CPU only: the source never touches
the GPU."""
import ctypes as C
import os
import time

import numpy as np
import pytest

from synth import configs


def _chunks():
    return [configs.blob_set(60, 40.0, 2, 0, start=20 * c, count=20) for c in range(3)] + \
        [configs.tube_set(3, 80.0, 2, 1, length_range=(50.0, 90.0))]


def _same(view, ms):
    assert view.n == ms.n and view.n_lods == ms.n_lods
    for l in range(ms.n_lods):
        assert np.array_equal(view.verts[l], ms.verts[l])
        assert np.array_equal(view.vert_off[l], ms.vert_off[l])
        assert np.array_equal(view.faces[l], ms.faces[l])
        if ms.face_off[l] is None:
            assert view.face_off[l] is None
        else:
            assert np.array_equal(view.face_off[l], ms.face_off[l])
        for a, b in ((view.hd[l], ms.hd[l]), (view.ph[l], ms.ph[l])):
            assert (a is None) == (b is None)
            if b is not None:
                assert np.array_equal(a, b)
    assert np.array_equal(view.anchor, ms.anchor)


@pytest.fixture
def files(tmp_path):
    from paper_2604_19982_gb300 import pj
    chunks = _chunks()
    paths = [str(tmp_path / f"c{c}.pjc") for c in range(len(chunks))]
    for p, ms in zip(paths, chunks):
        pj.write_chunk_file(p, ms)
    return pj, chunks, paths


@pytest.mark.parametrize("readahead", [0, 1, 2, 5])
def test_round_trip_over_passes(files, readahead):
    pj, chunks, paths = files
    src = pj.ChunkSource(paths, readahead)
    assert src.n_objects == sum(c.n for c in chunks) and src.n_chunks == len(chunks) and src.n_lods == 3
    for _ in range(3):      # every join over the set starts again at chunk 0
        for c, ms in enumerate(chunks):
            _same(src.chunk(c), ms)
    st = src.stats()
    assert st["restarts"] == 2 and st["chunks_read"] == 3 * len(chunks)
    assert st["bytes_read"] == 3 * sum(os.path.getsize(p) for p in paths)
    src.close()


def test_restart_in_the_middle(files):
    pj, chunks, paths = files
    src = pj.ChunkSource(paths, 1)
    _same(src.chunk(0), chunks[0])
    _same(src.chunk(1), chunks[1])
    _same(src.chunk(0), chunks[0])      # a cancelled join, then a new one
    for c in range(1, len(chunks)):
        _same(src.chunk(c), chunks[c])
    _same(src.chunk(2), chunks[2])      # a jump restarts at the chunk asked for
    assert src.stats()["restarts"] == 2
    src.close()


def test_reader_stays_within_its_buffers(files):
    pj, chunks, paths = files
    src = pj.ChunkSource(paths, 1)      # 3 buffers: chunks 0 and 1 before any request
    t = time.time()
    while src.stats()["chunks_read"] < 2 and time.time() - t < 10:
        time.sleep(0.01)
    time.sleep(0.2)
    assert src.stats()["chunks_read"] == 2
    src.chunk(0)                        # in use: 0; 1 read ahead; one buffer for the chunk before
    time.sleep(0.2)
    assert src.stats()["chunks_read"] == 2
    src.chunk(1)                        # in use: 0 and 1; 2 read ahead
    t = time.time()
    while src.stats()["chunks_read"] < 3 and time.time() - t < 10:
        time.sleep(0.01)
    time.sleep(0.2)
    assert src.stats()["chunks_read"] == 3
    src.close()


def test_fill_through_the_callback_pointer(files):
    # the pointer a streamed join calls from its loader threads
    pj, chunks, paths = files
    src = pj.ChunkSource(paths, 2)
    fill = C.cast(pj.lib().pj_chunk_source_fill, pj.FILL_FN)
    for c, ms in enumerate(chunks):
        d = pj.MeshSetDesc()
        assert fill(src.h, c, C.byref(d)) == pj.PJ_OK
        _same(pj.ChunkView(d), ms)
    d = pj.MeshSetDesc()
    assert fill(src.h, len(chunks), C.byref(d)) == pj.PJ_EINVAL
    assert fill(src.h, -1, C.byref(d)) == pj.PJ_EINVAL
    src.close()


def test_bad_files_are_reported(files, tmp_path):
    pj, chunks, paths = files
    missing = str(tmp_path / "absent.pjc")
    with pytest.raises(pj.PJError) as e:
        pj.ChunkSource([paths[0], missing])
    assert e.value.status == pj.PJ_ESOURCE
    raw = bytearray(open(paths[0], "rb").read())
    bad = tmp_path / "magic.pjc"
    bad.write_bytes(b"XX" + bytes(raw[2:]))
    short = tmp_path / "short.pjc"
    short.write_bytes(bytes(raw[:-64]))
    tiny = tmp_path / "tiny.pjc"
    tiny.write_bytes(bytes(raw[:100]))
    for p in (bad, short, tiny):
        with pytest.raises(pj.PJError) as e:
            pj.ChunkSource([str(p)])
        assert e.value.status == pj.PJ_EINVAL
    with pytest.raises(pj.PJError) as e:      # LoD counts differ
        two = configs.blob_set(3, 10.0, 1, 0, subs=(1, 2))
        p2 = str(tmp_path / "two.pjc")
        pj.write_chunk_file(p2, two)
        pj.ChunkSource([paths[0], p2])
    assert e.value.status == pj.PJ_EINVAL


def test_changed_file_is_reported_at_fill(files, tmp_path):
    pj, chunks, paths = files
    src = pj.ChunkSource(paths, 0)
    _same(src.chunk(0), chunks[0])
    pj.write_chunk_file(paths[2], chunks[3])   # replaced after opening
    with pytest.raises(pj.PJError) as e:
        src.chunk(1)
        src.chunk(2)
    assert e.value.status == pj.PJ_ESOURCE
    src.close()


def test_inconsistent_desc_is_not_written(tmp_path):
    from paper_2604_19982_gb300 import pj
    ms = configs.blob_set(4, 10.0, 1, 0)
    ms.vert_off[1] = ms.vert_off[1] + 1       # does not start at 0
    p = str(tmp_path / "x.pjc")
    with pytest.raises(pj.PJError) as e:
        pj.write_chunk_file(p, ms)
    assert e.value.status == pj.PJ_EINVAL
    assert not os.path.exists(p) and not os.path.exists(p + ".part")
