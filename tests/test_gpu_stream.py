"""Streamed joins (section 3.2, Algorithm 3; section 3.3, Algorithm 5): R arrives in chunks
through a fill callback while S stays resident.  A streamed join must
return exactly the pairs, brackets and distances of the same join over the
resident concatenation of the chunks (the per-pair schedule does not
depend on the other pairs), with R ids continuing across chunks; sampled
objects are also checked against the oracle.  Errors of the source stop
the join with the documented status."""
import numpy as np
import pytest

import oracle
from synth import configs
from synth.mesh import MeshSet

pytestmark = pytest.mark.gpu

SIDE = 150.0
N_R = 2400


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def data(ctx):
    """R: sub-3 blobs; S: 60 short tubes (2k-6k facets)."""
    R = configs.blob_set(N_R, SIDE, 7, 0)
    S = configs.tube_set(60, SIDE, 7, 1, length_range=(50.0, 120.0))
    return R, S, ctx.load_set(R), ctx.load_set(S)


@pytest.fixture(scope="module")
def blobs_s(ctx):
    S = configs.blob_set(N_R, SIDE, 7, 1)
    return S, ctx.load_set(S)


def chunk_of(start, count):
    return configs.blob_set(N_R, SIDE, 7, 0, start=start, count=count)


def bounds(sizes):
    b = np.concatenate([[0], np.cumsum(sizes)])
    return [(int(b[i]), int(b[i + 1] - b[i])) for i in range(len(sizes))]


def key(res):
    o = np.lexsort((res.s, res.r))
    return (res.r[o], res.s[o], res.d_lo[o], res.d_hi[o], res.d[o], res.exact[o])


def same(a, b):
    for x, y in zip(key(a), key(b)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("sizes", [[600, 600, 600, 600], [1000, 0, 1, 1399]])
def test_streamed_within_equals_resident(ctx, data, sizes):
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = data
    parts = bounds(sizes)
    gRs = ctx.load_set_streamed(N_R, len(parts), lambda c: chunk_of(*parts[c]))
    for prec, fl in ((pj.FP32, pj.TILE_PRUNE), (pj.FP32, pj.TILE_PRUNE | pj.EXACT_DIST), (pj.FP64, 0)):
        a = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=prec, flags=fl)
        b = ctx.join(gRs, gS, pj.WITHIN, tau=1.0, prec=prec, flags=fl)
        st = ctx.stats()
        assert st["streamed"] == 1 and st["chunks"] == len(parts) and st["objects"] == N_R
        assert st["bytes_h2d"] > 0
        assert a.n > 0
        same(a, b)
    gRs.free()


def test_streamed_oracle_sample(ctx, data, blobs_s):
    from paper_2604_19982_gb300 import pj
    R = data[0]
    S, gS = blobs_s
    parts = bounds([800, 800, 800])
    gRs = ctx.load_set_streamed(N_R, 3, lambda c: chunk_of(*parts[c]))
    res = ctx.join(gRs, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    hit = np.unique(res.r)
    rng = np.random.default_rng(3)
    rl = np.sort(np.concatenate([rng.choice(hit, min(4, len(hit)), replace=False),
                                 rng.choice(N_R, 4, replace=False)]))
    r, s, d = oracle.join_within(R, S, 1.0, rlist=rl)
    sel = np.isin(res.r, rl)
    got = sorted(zip(res.r[sel].tolist(), res.s[sel].tolist()))
    assert got == sorted(zip(r.tolist(), s.tolist()))
    dm = {(a, b): v for a, b, v in zip(r.tolist(), s.tolist(), d.tolist())}
    for a, b, v in zip(res.r[sel].tolist(), res.s[sel].tolist(), res.d[sel].tolist()):
        w = dm[(a, b)]
        assert abs(v - w) <= 1e-12 * max(w, 1.0)
    gRs.free()


def test_streamed_knn_equals_resident(ctx, data):
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = data
    parts = bounds([1200, 1200])
    gRs = ctx.load_set_streamed(N_R, 2, lambda c: chunk_of(*parts[c]))
    a = ctx.join(gR, gS, pj.KNN, k=2, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    b = ctx.join(gRs, gS, pj.KNN, k=2, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    assert a.n == b.n == 2 * N_R
    same(a, b)
    gRs.free()


def test_streamed_errors(ctx, data):
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = data
    parts = bounds([800, 800, 800])

    def cancel_at_1(c):
        if c == 1:
            raise pj.Cancel()
        return chunk_of(*parts[c])

    def broken(c):
        if c == 2:
            raise ValueError("source failed")
        return chunk_of(*parts[c])

    def wrong_lods(c):
        m = chunk_of(*parts[c])
        if c == 1:
            m = MeshSet(n=m.n, n_lods=2, verts=m.verts[1:], vert_off=m.vert_off[1:], faces=m.faces[1:],
                        face_off=m.face_off[1:], hd=m.hd[1:], ph=m.ph[1:], anchor=m.anchor, kind=m.kind)
        return m

    for fn, status in ((cancel_at_1, pj.PJ_ECANCELLED), (broken, pj.PJ_ESOURCE), (wrong_lods, pj.PJ_EINVAL)):
        g = ctx.load_set_streamed(N_R, 3, fn)
        with pytest.raises(pj.PJError) as e:
            ctx.join(g, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
        assert e.value.status == status
        g.free()
    # fewer objects than announced
    g = ctx.load_set_streamed(N_R + 5, 3, lambda c: chunk_of(*parts[c]))
    with pytest.raises(pj.PJError) as e:
        ctx.join(g, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
    assert e.value.status == pj.PJ_ESOURCE
    g.free()
    # the context stays usable
    res = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
    assert res.n > 0


def _pinned(ms):
    """The chunk's arrays in pinned host memory (page-locked by torch)."""
    import copy
    import torch
    out = copy.copy(ms)
    cache = {}

    def pin(a):
        if a is None:
            return None
        if id(a) not in cache:
            cache[id(a)] = torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        return cache[id(a)]

    for f in ("verts", "vert_off", "faces", "face_off", "hd", "ph"):
        setattr(out, f, [pin(a) for a in getattr(ms, f)])
    out.anchor = pin(ms.anchor)
    return out


def _on_device(ms):
    """verts, faces, hd, ph, anchor as CUDA tensors; offsets stay on the host."""
    import copy
    import torch
    out = copy.copy(ms)
    cache = {}

    def dev(a):
        if a is None:
            return None
        if id(a) not in cache:
            cache[id(a)] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        return cache[id(a)]

    for f in ("verts", "faces", "hd", "ph"):
        setattr(out, f, [dev(a) for a in getattr(ms, f)])
    out.anchor = dev(ms.anchor)
    return out


@pytest.mark.parametrize("where", ["pinned", "device"])
def test_streamed_pinned_and_device_chunks(ctx, data, where):
    """Chunks whose arrays already lie in pinned host memory are copied
    without packing (the arrays of the LoDs laid out on demand are read in
    place over the host link instead), and device arrays are read in place:
    the same result as the resident join, and only the host-side arrays
    travel."""
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = data
    parts = bounds([700, 900, 800])
    conv = _pinned if where == "pinned" else _on_device
    chunks = [conv(chunk_of(*p)) for p in parts]
    plain_chunks = [chunk_of(*p) for p in parts]
    g = ctx.load_set_streamed(N_R, 3, lambda c: chunks[c])
    gp = ctx.load_set_streamed(N_R, 3, lambda c: plain_chunks[c])
    for prec, fl in ((pj.FP32, pj.TILE_PRUNE), (pj.FP64, 0)):
        a = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=prec, flags=fl)
        ctx.join(gp, gS, pj.WITHIN, tau=1.0, prec=prec, flags=fl)
        packed_bytes = ctx.stats()["bytes_h2d"]
        b = ctx.join(g, gS, pj.WITHIN, tau=1.0, prec=prec, flags=fl)
        st = ctx.stats()
        same(a, b)
        if where == "pinned":
            # the same bytes without packing them, less those read in place
            assert st["bytes_host_read_max"] > 0
            assert st["bytes_h2d"] + st["bytes_host_read_max"] == packed_bytes
        else:
            assert st["bytes_h2d"] < packed_bytes / 20     # offsets only
    # the learned start reads every object's hd / ph maxima of those LoDs
    ctx.mlp_fit(gR, gS, pj.WITHIN, tau=1.0, max_pairs=20_000, epochs=3, seed=1)
    a = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.USE_MLP)
    b = ctx.join(g, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.USE_MLP)
    assert a.pairs() == b.pairs()
    g.free()
    gp.free()


def test_streamed_device_offsets_rejected(ctx, data):
    import copy
    import torch
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = data
    m = copy.copy(chunk_of(0, N_R))
    m.vert_off = [torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in m.vert_off]
    g = ctx.load_set_streamed(N_R, 1, lambda c: m)
    with pytest.raises(pj.PJError) as e:
        ctx.join(g, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
    assert e.value.status == pj.PJ_EINVAL
    g.free()
