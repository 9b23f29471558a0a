"""PJ_AUTOTUNE: the first join of a workload key tries every candidate
configuration (refinement variant x LoD schedule, then the unit tile of 16
and 8 s facets with the best of those) and keeps the fastest;
later joins reuse it, also from another context through the cache file.
Configurations only reschedule work, so the pairs must equal those of the
untuned join, and with PJ_EXACT_DIST every field (a pair confirmed at
another LoD step reports that step's bracket otherwise); both refinement
variants are also pinned directly through the "refine_variant" option."""

import numpy as np
import pytest

from synth import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sets():
    w = configs.blobs20k(n=2000)
    return w


def key(res):
    o = np.lexsort((res.s, res.r))
    return tuple(x[o] for x in (res.r, res.s, res.d_lo, res.d_hi, res.d, res.exact))


def same(a, b, exact=True):
    ka, kb = key(a), key(b)
    n = len(ka) if exact else 2
    for x, y in zip(ka[:n], kb[:n]):
        assert np.array_equal(x, y)


def test_autotune_within_and_cache_file(sets, tmp_path):
    from paper_2604_19982_gb300 import pj
    path = str(tmp_path / "tune.txt")
    ctx = pj.Context(0, {"autotune_cache": path})
    gR, gS = ctx.load_set(sets.R), ctx.load_set(sets.S)
    for tau, fl in ((0.0, pj.TILE_PRUNE), (1.0, pj.TILE_PRUNE | pj.EXACT_DIST)):
        ref = ctx.join(gR, gS, pj.WITHIN, tau=tau, prec=pj.FP32, flags=fl)
        a = ctx.join(gR, gS, pj.WITHIN, tau=tau, prec=pj.FP32, flags=fl | pj.AUTOTUNE)
        st = ctx.stats()["autotune"]
        # 2 variants x 3 start steps, then tiles of 16 and 8 s facets
        assert st["cached"] == 0 and len(st["tried"]) == 8
        assert [t["tile_s"] for t in st["tried"]] == [32] * 6 + [16, 8]
        assert st["tile_s"] in (32, 16, 8)
        best = [t for t in st["tried"] if t["tile_s"] == st["tile_s"] and t["variant"] == st["variant"]
                and t["start"] == st["start"]]
        assert best and best[0]["ms"] == min(t["ms"] for t in st["tried"] if "ms" in t)
        same(ref, a, fl & pj.EXACT_DIST)
        b = ctx.join(gR, gS, pj.WITHIN, tau=tau, prec=pj.FP32, flags=fl | pj.AUTOTUNE)
        assert ctx.stats()["autotune"]["cached"] == 1
        same(ref, b, fl & pj.EXACT_DIST)
    ctx.close()
    lines = open(path).read().split("\n")
    assert len([x for x in lines if x.strip()]) == 2
    ctx2 = pj.Context(0, {"autotune_cache": path})
    gR, gS = ctx2.load_set(sets.R), ctx2.load_set(sets.S)
    c = ctx2.join(gR, gS, pj.WITHIN, tau=0.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE)
    assert ctx2.stats()["autotune"]["cached"] == 1
    assert c.n > 0
    ctx2.close()


def test_autotune_keeps_fixed_variant(sets):
    """A refinement variant fixed at context creation is kept: only the
    LoD schedule is tuned, and the result equals the untuned join."""
    from paper_2604_19982_gb300 import pj
    ctx = pj.Context(0, {"refine_variant": 1})
    gR, gS = ctx.load_set(sets.R), ctx.load_set(sets.S)
    fl = pj.TILE_PRUNE | pj.EXACT_DIST
    ref = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl)
    a = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl | pj.AUTOTUNE)
    tried = ctx.stats()["autotune"]["tried"]
    assert len(tried) == 5 and all(t["variant"] == 1 for t in tried)
    same(ref, a)
    ctx.close()


def test_autotune_keeps_fixed_split(sets):
    """A unit split fixed at context creation is kept: no tile trials."""
    from paper_2604_19982_gb300 import pj
    ctx = pj.Context(0, {"refine_split": 2, "refine_tail": 64})
    gR, gS = ctx.load_set(sets.R), ctx.load_set(sets.S)
    fl = pj.TILE_PRUNE | pj.EXACT_DIST
    ref = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl)
    a = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=fl | pj.AUTOTUNE)
    tried = ctx.stats()["autotune"]["tried"]
    assert len(tried) == 6 and all(t["tile_s"] == 32 for t in tried)
    same(ref, a)
    ctx.close()


def test_autotune_knn_and_fp64(sets):
    from paper_2604_19982_gb300 import pj
    ctx = pj.Context(0)
    gR, gS = ctx.load_set(sets.R), ctx.load_set(sets.S)
    ref = ctx.join(gR, gS, pj.KNN, k=3, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    a = ctx.join(gR, gS, pj.KNN, k=3, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST | pj.AUTOTUNE)
    assert len(ctx.stats()["autotune"]["tried"]) == 4   # 2 variants, then 2 tiles
    same(ref, a)
    ref = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP64)
    a = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP64, flags=pj.AUTOTUNE)
    assert len(ctx.stats()["autotune"]["tried"]) == 5   # FP64: schedules, then tiles
    same(ref, a, exact=False)
    ctx.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_refine_variants_agree(sets, variant):
    from paper_2604_19982_gb300 import pj
    base = pj.Context(0)
    ctx = pj.Context(0, {"refine_variant": variant})
    out = []
    for c in (base, ctx):
        gR, gS = c.load_set(sets.R), c.load_set(sets.S)
        out.append([c.join(gR, gS, pj.WITHIN, tau=t, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
                    for t in (0.0, 1.0)])
    for a, b in zip(*out):
        assert np.array_equal(np.sort(a.r * 100000 + a.s), np.sort(b.r * 100000 + b.s))
        same(a, b)
    base.close()
    ctx.close()
    with pytest.raises(pj.PJError):
        pj.Context(0, {"refine_variant": 3})


@pytest.mark.parametrize("opts", [{"refine_split": 1}, {"refine_split": 2, "refine_tail": 64},
                                  {"refine_split": 8, "refine_tail": 64},
                                  {"refine_split": 4, "refine_tail": 64, "refine_variant": 2}])
def test_tail_split_agrees(sets, opts):
    """Splitting the last units (here: all of them) into parts over their s
    facets only reschedules the refinement: the same pairs, and with
    PJ_EXACT_DIST the same fields, for within and k-NN joins."""
    from paper_2604_19982_gb300 import pj
    base = pj.Context(0, {"refine_split": 1})
    ctx = pj.Context(0, opts)
    out = []
    for c in (base, ctx):
        gR, gS = c.load_set(sets.R), c.load_set(sets.S)
        out.append([c.join(gR, gS, pj.WITHIN, tau=t, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
                    for t in (0.0, 1.0)]
                   + [c.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE),
                      c.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP64, flags=pj.TILE_PRUNE | pj.EXACT_DIST),
                      c.join(gR, gS, pj.KNN, k=3, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)])
    for i, (a, b) in enumerate(zip(*out)):
        same(a, b, exact=(i != 2))
    base.close()
    ctx.close()
    for bad in ({"refine_split": 3}, {"refine_tail": -1}):
        with pytest.raises(pj.PJError):
            pj.Context(0, bad)


def test_autotune_streamed(sets):
    from paper_2604_19982_gb300 import pj
    ctx = pj.Context(0)
    gR, gS = ctx.load_set(sets.R), ctx.load_set(sets.S)
    ref = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    parts = [(0, 1000), (1000, 1000)]
    g = ctx.load_set_streamed(2000, 2, lambda c: configs.blob_set(2000, sets_side(), 0, 0, start=parts[c][0],
                                                                  count=parts[c][1]))
    a = ctx.join(g, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST | pj.AUTOTUNE)
    same(ref, a)
    ctx.close()


def sets_side():
    return configs.scaled_side(400.0, 20_000, 2000)
