"""Uneven workloads: vessel-like tubes (per-object topology, thousands to
tens of thousands of facets) against nucleus blobs, within tau = 2.  Every
precision / pruning mode must return the same pairs.  The oracle pins them
on samples it can afford: for tube objects r, sampled pairs (result pairs
and near misses whose boxes are within tau, chosen from the inputs and the
FP64 result alone) get their exact distance, which must fall on the right
side of tau and, with PJ_EXACT_DIST, match within 1e-12 relative; for
blob objects r (few candidate tubes each), the full result of sampled r is
compared.  The full workload (2,000 tubes x 200,000 blobs) is checked the
same way."""
import numpy as np
import pytest

import oracle
from synth import configs

pytestmark = pytest.mark.gpu

SIDE = 120.0
TAU = 2.0


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small(ctx):
    R = configs.tube_set(40, SIDE, 3, 0, length_range=(50.0, 120.0))
    S = configs.blob_set(3000, SIDE, 3, 1)
    return R, S, ctx.load_set(R), ctx.load_set(S)


def pairs(res):
    return sorted(zip(res.r.tolist(), res.s.tolist()))


def check_oracle(res, R, S, tau, rl, exact):
    """Full result of the objects rl of R against the oracle."""
    r, s, d = oracle.join_within(R, S, tau, rlist=np.sort(rl))
    sel = np.isin(res.r, rl)
    got = sorted(zip(res.r[sel].tolist(), res.s[sel].tolist()))
    assert got == sorted(zip(r.tolist(), s.tolist()))
    want = {(a, b): v for a, b, v in zip(r.tolist(), s.tolist(), d.tolist())}
    for a, b, lo, hi, dv, ex in zip(res.r[sel].tolist(), res.s[sel].tolist(), res.d_lo[sel].tolist(),
                                    res.d_hi[sel].tolist(), res.d[sel].tolist(), res.exact[sel].tolist()):
        w = want[(a, b)]
        assert lo <= w + 1e-12 * max(w, 1.0) and w <= hi + 1e-12 * max(w, 1.0)
        if exact:
            assert ex == 1 and abs(dv - w) <= 1e-12 * max(w, 1e-300)


def box_candidates(R, S, tau):
    """Pairs whose boxes are within tau (numpy, from the meshes alone)."""
    a, b = R.mbb().astype(np.float64), S.mbb().astype(np.float64)
    out = []
    for r in range(R.n):
        g = np.maximum(0, np.maximum(b[:, :3] - a[r, 3:], a[r, :3] - b[:, 3:]))
        for s in np.nonzero((g * g).sum(1) <= tau * tau)[0]:
            out.append((r, int(s)))
    return out


def check_pairs(res, R, S, tau, k, seed):
    """k result pairs and k near misses: exact distances by the oracle."""
    rng = np.random.default_rng(seed)
    got = {(a, b): (dv, ex) for a, b, dv, ex in zip(res.r.tolist(), res.s.tolist(), res.d.tolist(),
                                                   res.exact.tolist())}
    hits = sorted(got)
    miss = [p for p in box_candidates(R, S, tau) if p not in got]
    pick = [hits[i] for i in rng.choice(len(hits), min(k, len(hits)), replace=False)]
    pick += [miss[i] for i in rng.choice(len(miss), min(k, len(miss)), replace=False)]
    pr = np.array([p[0] for p in pick], np.int32)
    ps = np.array([p[1] for p in pick], np.int32)
    d = oracle.pair_dists(R, S, pr, ps)
    for (a, b), w in zip(pick, d.tolist()):
        if (a, b) in got:
            assert w <= tau
            dv, ex = got[(a, b)]
            if ex == 1:
                assert abs(dv - w) <= 1e-12 * max(w, 1e-300)
        else:
            assert w > tau


MODES = {
    "fp64": dict(prec=0, flags=0),
    "fp32": dict(prec=1, flags=0),
    "fp32_prune": dict(prec=1, flags=16),
    "fp32_prune_exact": dict(prec=1, flags=16 | 1),
}


def test_tubes_vs_blobs_all_modes(ctx, small):
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = small
    out = {m: ctx.join(gR, gS, pj.WITHIN, tau=TAU, **kw) for m, kw in MODES.items()}
    ref = pairs(out["fp64"])
    assert len(ref) > 0
    for m, res in out.items():
        assert pairs(res) == ref, m
    check_pairs(out["fp32_prune_exact"], R, S, TAU, 6, 1)


def test_blobs_vs_tubes(ctx, small):
    """Roles swapped: R blobs, S tubes (the layout of the streamed workload)."""
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = small
    a = ctx.join(gS, gR, pj.WITHIN, tau=TAU, prec=pj.FP64)
    b = ctx.join(gS, gR, pj.WITHIN, tau=TAU, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    assert pairs(a) == pairs(b) and a.n > 0
    hit = np.unique(b.r)
    rl = np.unique(np.concatenate([hit[:4], [5, 6]]))
    check_oracle(b, S, R, TAU, rl, exact=True)


def test_tubes_knn(ctx, small):
    """k-NN both ways: tubes' nearest blobs (precision modes agree) and
    blobs' nearest tubes (also against the oracle on sampled blobs)."""
    from paper_2604_19982_gb300 import pj
    R, S, gR, gS = small
    a = ctx.join(gR, gS, pj.KNN, k=2, prec=pj.FP64)
    b = ctx.join(gR, gS, pj.KNN, k=2, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    assert a.n == b.n == 2 * R.n
    assert pairs(a) == pairs(b)
    c = ctx.join(gS, gR, pj.KNN, k=2, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    assert c.n == 2 * S.n
    rl = np.array([3, 700, 2100])
    r, s, d = oracle.join_knn(S, R, 2, rlist=rl)
    sel = np.isin(c.r, rl)
    assert sorted(zip(c.r[sel].tolist(), c.s[sel].tolist())) == sorted(zip(r.tolist(), s.tolist()))
    want = {(x, y): v for x, y, v in zip(r.tolist(), s.tolist(), d.tolist())}
    for x, y, dv in zip(c.r[sel].tolist(), c.s[sel].tolist(), c.d[sel].tolist()):
        assert abs(dv - want[(x, y)]) <= 1e-12 * max(want[(x, y)], 1e-300)


def test_full_size_tubes2k_sampled(ctx):
    """2,000 tubes x 200,000 blobs, side 2,320, tau = 2."""
    from paper_2604_19982_gb300 import pj
    w = configs.tubes2k()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    a = ctx.join(gR, gS, pj.WITHIN, tau=TAU, prec=pj.FP32, flags=pj.TILE_PRUNE)
    b = ctx.join(gR, gS, pj.WITHIN, tau=TAU, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    assert pairs(a) == pairs(b) and a.n > 0
    assert np.all(b.exact == 1) and np.all(b.d <= TAU)
    check_pairs(b, w.R, w.S, TAU, 6, 2)
    gR.free()
    gS.free()


def test_unit_buffer_overflow_reruns_with_equal_results():
    """With a unit budget of 1 MB (32,768 units), tube joins overflow the
    unit buffer; the join grows it to the count needed and runs again: the
    results equal those of a context with the default budget."""
    from paper_2604_19982_gb300 import pj
    R = configs.tube_set(80, 300.0, 3, 0, length_range=(50.0, 200.0))
    S = configs.blob_set(6000, 300.0, 3, 1)
    out = []
    for opts in ({}, {"unit_budget_mb": 1}):
        c = pj.Context(0, opts)
        gR, gS = c.load_set(R), c.load_set(S)
        # no unit pruning: every block pair of a candidate is a unit, so the
        # coarse step needs far more than the small budget's 32,768 units
        res = c.join(gR, gS, pj.WITHIN, tau=2.0, prec=pj.FP32, flags=0)
        again = c.join(gR, gS, pj.WITHIN, tau=2.0, prec=pj.FP32, flags=0)
        out.append((res, again, c.stats()))
        c.close()
    (a, _, _), (b, b2, st) = out
    assert a.n > 0
    for x in (b, b2):
        assert x.pairs() == a.pairs()
        assert np.array_equal(x.d_lo, a.d_lo) and np.array_equal(x.d_hi, a.d_hi)
    # the small budget was really exceeded at some step
    assert max(x["tiles"] for x in st["steps"]) > 32768
