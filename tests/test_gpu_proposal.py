"""The learned proposal inside the joins.  It only reorders work (k-NN
first waves) or skips coarse steps (within-tau start LoD), so a join with
PJ_USE_MLP must return exactly the pairs of the same join without it, and
on the clustered k-NN workload (50,000 x 50,000 sub-3 blobs, 20-cluster
mixture, k = 3) weights fitted on the seed-1 run must save triangle tests
on the seed-0 run."""
import numpy as np
import pytest

import oracle
from synth import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


def pairs(res):
    return sorted(zip(res.r.tolist(), res.s.tolist()))


def test_join_without_weights_fails(ctx):
    from paper_2604_19982_gb300 import pj
    w = configs.blobs100()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    fresh = pj.Context(0)
    gR2, gS2 = fresh.load_set(w.R), fresh.load_set(w.S)
    with pytest.raises(pj.PJError):
        fresh.join(gR2, gS2, pj.KNN, k=2, prec=pj.FP32, flags=pj.USE_MLP)
    fresh.close()
    gR.free()
    gS.free()


def test_fit_rejects_bad_queries(ctx):
    from paper_2604_19982_gb300 import pj
    w = configs.blobs100()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    with pytest.raises(pj.PJError):
        ctx.mlp_fit(gR, gS, pj.KNN, k=0)
    with pytest.raises(pj.PJError):
        ctx.mlp_fit(gR, gS, pj.WITHIN, tau=-1.0)
    with pytest.raises(pj.PJError):
        ctx.mlp_fit(gR, gS, pj.KNN, k=3, max_pairs=8)
    gR.free()
    gS.free()


def test_within_small_same_pairs(ctx):
    """blobs100, tau = 0.5: fit on seed 1, then every precision with and
    without the proposal against the oracle."""
    from paper_2604_19982_gb300 import pj
    w1 = configs.blobs100(seed=1)
    g1R, g1S = ctx.load_set(w1.R), ctx.load_set(w1.S)
    rmse = ctx.mlp_fit(g1R, g1S, pj.WITHIN, tau=2.0, epochs=80, seed=1)
    assert np.isfinite(rmse) and rmse < 0.5
    g1R.free()
    g1S.free()
    w = configs.blobs100()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    r, s, _ = oracle.join_within(w.R, w.S, 0.5)
    want = sorted(zip(r.tolist(), s.tolist()))
    for prec, fl in ((pj.FP64, 0), (pj.FP32, pj.TILE_PRUNE), (pj.FP32, pj.TILE_PRUNE | pj.EXACT_DIST)):
        a = ctx.join(gR, gS, pj.WITHIN, tau=0.5, prec=prec, flags=fl)
        b = ctx.join(gR, gS, pj.WITHIN, tau=0.5, prec=prec, flags=fl | pj.USE_MLP)
        assert ctx.stats()["mlp"] == 1
        assert pairs(a) == want and pairs(b) == want
        if fl & pj.EXACT_DIST:
            assert np.array_equal(a.d, b.d)
    gR.free()
    gS.free()


def test_knn_gain_clustered(ctx):
    from paper_2604_19982_gb300 import pj
    w1 = configs.knn50k(seed=1)
    g1R, g1S = ctx.load_set(w1.R), ctx.load_set(w1.S)
    rmse = ctx.mlp_fit(g1R, g1S, pj.KNN, k=3, max_pairs=200000, epochs=30, seed=1)
    assert rmse < 0.15, rmse
    g1R.free()
    g1S.free()
    w = configs.knn50k()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    a = ctx.join(gR, gS, pj.KNN, k=3, prec=pj.FP32, flags=pj.TILE_PRUNE)
    sa = ctx.stats()
    b = ctx.join(gR, gS, pj.KNN, k=3, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.USE_MLP)
    sb = ctx.stats()
    assert a.n == b.n == 3 * w.R.n
    assert pairs(a) == pairs(b)
    ta = sa["tests_fp32"] + sa["tests_fp64"]
    tb = sb["tests_fp32"] + sb["tests_fp64"]
    assert tb < 0.98 * ta, (ta, tb)
    rl = np.sort(np.random.default_rng(5).choice(w.R.n, 12, replace=False))
    r, s, _ = oracle.join_knn(w.R, w.S, 3, rlist=rl)
    sel = set(rl.tolist())
    got = sorted((x, y) for x, y in pairs(b) if x in sel)
    assert got == sorted(zip(r.tolist(), s.tolist()))
    gR.free()
    gS.free()
