"""k-NN join (Algorithm 6, corrected reading) through the C ABI against the
oracle.  For every r the set of its min(k, |S|) neighbours must equal the
oracle's (ids bit-exact; ties broken by the id of s).  Without
PJ_EXACT_DIST the neighbours come ordered by s and each oracle distance must
lie in the reported bracket; with it they come ordered by (d, s) with FP64
distances within 1e-12 relative."""
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


def check_knn(res, R, S, k, rlist=None, exact_order=False):
    r, s, d = oracle.join_knn(R, S, k, rlist=rlist)
    want = {}
    for a, b, dd in zip(r.tolist(), s.tolist(), d.tolist()):
        want.setdefault(a, []).append((b, dd))
    got = {}
    for i in range(res.n):
        got.setdefault(int(res.r[i]), []).append(i)
    rs = rlist if rlist is not None else range(R.n)
    for rr in rs:
        rr = int(rr)
        w = want.get(rr, [])
        g = got.get(rr, [])
        assert sorted(x for x, _ in w) == sorted(int(res.s[i]) for i in g), f"r={rr}"
        dmap = dict(w)
        for i in g:
            dv = dmap[int(res.s[i])]
            slack = 1e-12 * max(dv, 1.0)
            assert res.d_lo[i] <= dv + slack and dv <= res.d_hi[i] + slack, f"r={rr} bracket"
        if exact_order:
            assert [int(res.s[i]) for i in g] == [x for x, _ in w], f"r={rr} order"
            for i in g:
                dv = dmap[int(res.s[i])]
                assert res.exact[i] == 1 and abs(res.d[i] - dv) <= 1e-12 * dv, f"r={rr} distance"
    assert set(got) <= set(int(x) for x in rs) or rlist is not None


MODES = {
    "fp64": dict(prec=0, flags=0),
    "fp32": dict(prec=1, flags=0),
    "fp32_prune": dict(prec=1, flags=16),
}


@pytest.fixture(scope="module")
def small(ctx):
    w = configs.blobs100()
    return w, ctx.load_set(w.R), ctx.load_set(w.S)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("k", [1, 3])
def test_knn_blobs100(ctx, small, mode, k):
    from paper_2604_19982_gb300 import pj
    w, gR, gS = small
    res = ctx.join(gR, gS, pj.KNN, k=k, **MODES[mode])
    assert res.n == w.R.n * k
    check_knn(res, w.R, w.S, k)


def test_knn_exact_order(ctx, small):
    from paper_2604_19982_gb300 import pj
    w, gR, gS = small
    res = ctx.join(gR, gS, pj.KNN, k=4, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    check_knn(res, w.R, w.S, 4, exact_order=True)


def test_knn_more_neighbours_than_objects(ctx, small):
    from paper_2604_19982_gb300 import pj
    w, gR, _ = small
    S2 = configs.blob_set(3, 20.0, 8, 1, subs=(1, 2))
    g2 = ctx.load_set(S2)
    res = ctx.join(gR, g2, pj.KNN, k=5, prec=pj.FP32, flags=pj.TILE_PRUNE)
    assert res.n == w.R.n * 3
    check_knn(res, w.R, S2, 5, rlist=np.arange(0, 100, 10))
    g2.free()


def test_knn_gmm_clusters(ctx):
    """Clustered centres (Gaussian mixture, sigma 15) as in the k-NN workload,
    1,500 objects per set, sampled objects r."""
    from paper_2604_19982_gb300 import pj
    gmm = configs.gmm_centres(0, 20, 1000.0)
    R = configs.blob_set(1500, 1000.0, 0, 0, subs=(1, 2), gmm=gmm)
    S = configs.blob_set(1500, 1000.0, 0, 1, subs=(1, 2), gmm=gmm)
    gR, gS = ctx.load_set(R), ctx.load_set(S)
    rl = np.random.default_rng(1).choice(R.n, 60, replace=False)
    for mode in ("fp64", "fp32_prune"):
        res = ctx.join(gR, gS, pj.KNN, k=3, **MODES[mode])
        check_knn(res, R, S, 3, rlist=np.sort(rl))
    gR.free()
    gS.free()
