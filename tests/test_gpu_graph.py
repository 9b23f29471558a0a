"""PJ_USE_GRAPH: after the filter, a within-tau join runs as one captured
CUDA graph per (sets, query, candidate capacity); the candidate list is
padded to a power of two with pairs marked REMOVED.  A replayed join must
return exactly what the direct join returns, for resident sets, every
precision, a changed query, and streamed chunks (whose slots alternate)."""
import numpy as np
import pytest

from synth import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def sets(ctx):
    w = configs.blobs20k(n=4000)
    return w, ctx.load_set(w.R), ctx.load_set(w.S)


def key(res):
    o = np.lexsort((res.s, res.r))
    return tuple(x[o] for x in (res.r, res.s, res.d_lo, res.d_hi, res.d, res.exact))


def same(a, b):
    for x, y in zip(key(a), key(b)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec,flags", [(1, 16), (1, 16 | 1), (0, 0), (1, 0)])
def test_graph_replay_equals_direct(ctx, sets, prec, flags):
    from paper_2604_19982_gb300 import pj
    w, gR, gS = sets
    for tau in (0.0, 1.0):
        ref = ctx.join(gR, gS, pj.WITHIN, tau=tau, prec=prec, flags=flags)
        modes, launches = [], []
        for _ in range(3):
            res = ctx.join(gR, gS, pj.WITHIN, tau=tau, prec=prec, flags=flags | pj.USE_GRAPH)
            st = ctx.stats()
            modes.append(st["graph"])
            launches.append(st["launches"])
            assert st["candidates"] <= st["capacity"]
            same(ref, res)
        assert modes[0] == "captured" and modes[1:] == ["replay", "replay"]
        assert launches[1] == launches[2] == launches[0]   # the graph holds the direct run's kernels


def test_graph_with_autotune_and_timeout(ctx, sets):
    from paper_2604_19982_gb300 import pj
    w, gR, gS = sets
    ref = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    for _ in range(2):
        res = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32,
                       flags=pj.TILE_PRUNE | pj.EXACT_DIST | pj.USE_GRAPH | pj.AUTOTUNE)
        same(ref, res)
    res = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST | pj.USE_GRAPH,
                   timeout_s=30.0)
    same(ref, res)


def test_graph_streamed_chunks(ctx, sets):
    from paper_2604_19982_gb300 import pj
    w, gR, gS = sets
    side = configs.scaled_side(400.0, 20_000, 4000)
    ref = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    parts = [(a, 500) for a in range(0, 4000, 500)]
    g = ctx.load_set_streamed(4000, len(parts), lambda c: configs.blob_set(4000, side, 0, 0, start=parts[c][0],
                                                                           count=parts[c][1]))
    for _ in range(2):
        res = ctx.join(g, gS, pj.WITHIN, tau=1.0, prec=pj.FP32,
                       flags=pj.TILE_PRUNE | pj.EXACT_DIST | pj.USE_GRAPH)
        same(ref, res)
    g.free()


@pytest.mark.parametrize("overlap", [0, 1])
def test_graph_streamed_speculative(sets, overlap):
    """After the first chunk of a streamed R on a join context, a chunk's
    whole join (filter included) runs as one graph with the capacity of the
    context's last chunk; a chunk with more pairs than that capacity runs
    again unspeculated.  With chunk_overlap the chunks alternate between the
    context and its twin (two joins in flight), each with its own grid and
    capacity.  Either way the result equals the resident join of the same
    objects."""
    from paper_2604_19982_gb300 import pj
    from synth.mesh import concat
    w, _, _ = sets
    c = pj.Context(0, {"chunk_overlap": overlap})
    gS = c.load_set(w.S)
    side = configs.scaled_side(400.0, 20_000, 4000)
    # chunks 0-2: blobs placed like S's, some tens of candidate pairs each;
    # chunk 3: copies of S's first 400 blobs (every one meets its copy), more
    # pairs than the capacity speculated from the earlier chunks
    parts = [configs.blob_set(400, side, 5, 0), configs.blob_set(400, side, 6, 0),
             configs.blob_set(400, side, 7, 0), configs.blob_set(4000, side, 0, 1, start=0, count=400)]
    whole = concat(parts)
    gW = c.load_set(whole)
    fl = pj.TILE_PRUNE | pj.EXACT_DIST
    ref = c.join(gW, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl)
    g = c.load_set_streamed(whole.n, len(parts), lambda i: parts[i])
    for i in range(3):
        res = c.join(g, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl | pj.USE_GRAPH)
        st = c.stats()
        same(ref, res)
        if i == 0:
            # the first chunk of each join context runs unspeculated; chunk 3
            # exceeds the capacity speculated from its context's first chunk
            assert st["spec_joins"] == (1 if overlap else 2) and st["spec_misses"] == 1
        else:
            # every chunk speculated; by the third join every graph is captured
            assert st["spec_joins"] == 4 and st["spec_misses"] == 0
            assert st["graph_replays"] == 4 or i == 1
    g.free()
    gW.free()
    gS.free()
    c.close()


def test_graph_flag_ignored_for_knn(ctx, sets):
    from paper_2604_19982_gb300 import pj
    w, gR, gS = sets
    a = ctx.join(gR, gS, pj.KNN, k=2, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    b = ctx.join(gR, gS, pj.KNN, k=2, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST | pj.USE_GRAPH)
    same(a, b)


def test_graph_with_learned_start(ctx, sets):
    """The learned start inside the captured sequence: the feature kernel
    skips the padding rows (no pair ids there), replay equals direct."""
    from paper_2604_19982_gb300 import pj
    w, gR, gS = sets
    ctx.mlp_fit(gR, gS, pj.WITHIN, tau=1.0, max_pairs=20_000, epochs=5, seed=1)
    fl = pj.TILE_PRUNE | pj.USE_MLP
    ref = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl)
    plain = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
    assert ref.pairs() == plain.pairs()   # the start step changes no result
    modes = []
    for _ in range(3):
        res = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl | pj.USE_GRAPH)
        modes.append(ctx.stats()["graph"])
        assert ctx.stats()["candidates"] < ctx.stats()["capacity"]
        same(ref, res)
    assert modes == ["captured", "replay", "replay"]
