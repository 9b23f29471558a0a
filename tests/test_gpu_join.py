"""Joins through the C ABI against the CPU oracle.

Pair sets must be identical (bit-exact ids, same order).  Distances:
exact == 1 (FP64 full resolution) within 1e-12 relative; exact == 2 (FP32
full resolution) within 1e-5 relative and the oracle inside [d_lo, d_hi];
exact == 0 (decided early) the oracle inside [d_lo, d_hi].
"""
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


def check_within(res, R, S, tau, rlist=None, oracle_out=None):
    r, s, d = oracle_out if oracle_out is not None else oracle.join_within(R, S, tau, rlist=rlist)
    got_r, got_s = res.r, res.s
    if rlist is not None:
        keep = np.isin(got_r, rlist)
        order = {int(x): i for i, x in enumerate(rlist)}
        idx = np.nonzero(keep)[0]
        idx = idx[np.lexsort((got_s[idx], [order[int(x)] for x in got_r[idx]]))]
        got = list(zip(got_r[idx].tolist(), got_s[idx].tolist()))
        sub = lambda a: a[idx]  # noqa: E731
    else:
        got = res.pairs()
        sub = lambda a: a  # noqa: E731
    assert got == list(zip(r.tolist(), s.tolist()))
    dlo, dhi, dd, ex = sub(res.d_lo), sub(res.d_hi), sub(res.d), sub(res.exact)
    slack = 1e-12 * np.maximum(d, 1.0)
    assert (dlo <= d + slack).all() and (d <= dhi + slack).all(), "oracle distance outside the bracket"
    e1 = ex == 1
    if e1.any():
        assert (np.abs(dd[e1] - d[e1]) <= 1e-12 * d[e1]).all() and ((dd[e1] == 0) == (d[e1] == 0)).all()
    e2 = ex == 2
    if e2.any():
        assert (np.abs(dd[e2] - d[e2]) <= 1e-5 * d[e2]).all()
    return ex


MODES = {
    "fp64": dict(prec=0, flags=0),
    "fp32": dict(prec=1, flags=0),
    "fp32_prune": dict(prec=1, flags=16),
    "fp32_prune_exact": dict(prec=1, flags=16 | 1),
    "fp64_exact": dict(prec=0, flags=1),
}


@pytest.fixture(scope="module")
def small(ctx):
    w = configs.blobs100()
    return w, ctx.load_set(w.R), ctx.load_set(w.S), oracle.join_within(w.R, w.S, 0.5)


@pytest.mark.parametrize("mode", list(MODES))
def test_blobs100_within(ctx, small, mode):
    from paper_2604_19982_gb300 import pj
    w, gR, gS, ref = small
    res = ctx.join(gR, gS, pj.WITHIN, tau=0.5, **MODES[mode])
    ex = check_within(res, w.R, w.S, 0.5, oracle_out=ref)
    if "exact" in mode:
        assert (ex == 1).all()
    st = ctx.stats()
    assert st["candidates"] >= res.n


def test_blobs100_intersection_and_tau_sweep(ctx, small):
    from paper_2604_19982_gb300 import pj
    w, gR, gS, _ = small
    res = ctx.join(gR, gS, pj.INTERSECT, prec=pj.FP32, flags=pj.TILE_PRUNE)
    check_within(res, w.R, w.S, 0.0)
    assert (res.d == 0).all() and res.n > 0
    prev = set()
    for tau in (0.0, 0.3, 1.0, 2.0):
        res = ctx.join(gR, gS, pj.WITHIN, tau=tau, prec=pj.FP32, flags=pj.TILE_PRUNE)
        cur = set(res.pairs())
        assert prev <= cur
        prev = cur
    check_within(res, w.R, w.S, 2.0)


def test_deterministic_and_symmetric(ctx, small):
    from paper_2604_19982_gb300 import pj
    w, gR, gS, _ = small
    a = ctx.join(gR, gS, pj.WITHIN, tau=0.5, prec=pj.FP32, flags=pj.TILE_PRUNE)
    b = ctx.join(gR, gS, pj.WITHIN, tau=0.5, prec=pj.FP32, flags=pj.TILE_PRUNE)
    assert a.pairs() == b.pairs()
    assert np.array_equal(a.d, b.d) and np.array_equal(a.d_lo, b.d_lo)
    t = ctx.join(gS, gR, pj.WITHIN, tau=0.5, prec=pj.FP64)
    assert sorted(a.pairs()) == sorted(zip(t.s.tolist(), t.r.tolist()))


@pytest.mark.parametrize("tau", [0.0, 1.0])
@pytest.mark.parametrize("mode", ["fp64", "fp32_prune"])
def test_blobs1000(ctx, tau, mode):
    from paper_2604_19982_gb300 import pj
    w = configs.blobs20k(n=1000)
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    res = ctx.join(gR, gS, pj.WITHIN, tau=tau, **MODES[mode])
    check_within(res, w.R, w.S, tau)
    gR.free()
    gS.free()


def test_full_size_blobs20k_sampled(ctx):
    """The benchmark's workload (20,000 x 20,000 sub-3 blobs, tau = 1): every
    result of a sample of objects r against the oracle."""
    from paper_2604_19982_gb300 import pj
    w = configs.blobs20k()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    res = ctx.join(gR, gS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
    rng = np.random.default_rng(0)
    have = np.unique(res.r)
    rl = np.unique(np.concatenate([rng.choice(have, min(25, len(have)), replace=False),
                                   rng.choice(w.R.n, 25, replace=False)]))
    check_within(res, w.R, w.S, 1.0, rlist=rl)
    res0 = ctx.join(gR, gS, pj.INTERSECT, prec=pj.FP32, flags=pj.TILE_PRUNE)
    have0 = np.unique(res0.r)
    rl0 = np.unique(np.concatenate([rng.choice(have0, min(25, len(have0)), replace=False),
                                    rng.choice(w.R.n, 25, replace=False)]))
    check_within(res0, w.R, w.S, 0.0, rlist=rl0)
    gR.free()
    gS.free()


def test_edge_cases(ctx, small):
    from paper_2604_19982_gb300 import pj
    w, gR, gS, _ = small
    empty = configs.blob_set(0, 10.0, 0, 0, subs=(1, 2))
    gE = ctx.load_set(empty)
    assert ctx.join(gE, gS, pj.WITHIN, tau=1.0).n == 0
    assert ctx.join(gR, gE, pj.WITHIN, tau=1.0, prec=pj.FP32).n == 0
    # far apart: no candidates at all
    far = configs.blob_set(5, 10.0, 9, 0, subs=(1, 2))
    far.verts = [v + np.float32(1e4) for v in far.verts]
    far.anchor = far.anchor + np.float32(1e4)
    gF = ctx.load_set(far)
    assert ctx.join(gF, gS, pj.WITHIN, tau=0.5).n == 0
    # a set against itself: every object meets itself
    res = ctx.join(gR, gR, pj.INTERSECT, prec=pj.FP32, flags=pj.TILE_PRUNE)
    assert set((i, i) for i in range(w.R.n)) <= set(res.pairs())
    # huge tau: every pair is a result, decided from anchors / coarse LoDs
    one = configs.blob_set(3, 5.0, 4, 0, subs=(1, 2))
    g1 = ctx.load_set(one)
    res = ctx.join(g1, g1, pj.WITHIN, tau=100.0, prec=pj.FP32)
    assert res.n == 9
    for s in (gE, gF, g1):
        s.free()


def test_errors_leave_context_usable(ctx, small):
    from paper_2604_19982_gb300 import pj
    w, gR, gS, ref = small
    with pytest.raises(pj.PJError) as e:
        ctx.join(gR, gS, pj.WITHIN, tau=0.5, timeout_s=1e-9)
    assert e.value.status == pj.PJ_ETIMEOUT
    with pytest.raises(pj.PJError) as e:
        ctx.join(gR, gS, pj.WITHIN, tau=-1.0)
    assert e.value.status == pj.PJ_EINVAL
    bad = configs.blob_set(2, 5.0, 1, 0, subs=(1, 2))
    bad.verts = [v.copy() for v in bad.verts]
    bad.verts[1][5, 1] = np.nan
    with pytest.raises(pj.PJError) as e:
        ctx.load_set(bad)
    assert e.value.status == pj.PJ_ENONFINITE
    bad2 = configs.blob_set(2, 5.0, 1, 0, subs=(1, 2))
    bad2.faces = [f.copy() for f in bad2.faces]
    bad2.faces[0][3, 2] = 10_000
    with pytest.raises(pj.PJError) as e:
        ctx.load_set(bad2)
    assert e.value.status == pj.PJ_EBOUNDS
    res = ctx.join(gR, gS, pj.WITHIN, tau=0.5, prec=pj.FP32, flags=pj.TILE_PRUNE)
    check_within(res, w.R, w.S, 0.5, oracle_out=ref)
