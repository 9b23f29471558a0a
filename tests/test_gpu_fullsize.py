"""Parity at the full sizes of the k-NN, vessel-nuclei and streaming
workloads: every result of sampled objects r (all of their candidates, not
a sample of pairs) against the oracle.

* knn50k: 50,000 x 50,000 clustered blobs, k = 3; the neighbour lists of
  120 objects r;
* tubes2k: 2,000 tubes x 200,000 blobs, tau = 2; each sampled tube's full
  result set, from the oracle's distances of every blob whose box lies
  within tau of the tube's;
* stream2m: two of the 64 chunks of the 2,000,000 streamed blobs against
  all 20,000 tubes, tau = 1; the full result sets of sampled blobs of both
  chunks.

The oracle's work is bounded by the sample (short tubes for tubes2k, a few
blobs per chunk for stream2m), the GPU runs the whole workload.
"""
import os

import numpy as np
import pytest

import oracle
from synth import configs
from synth.mesh import concat, subset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


def _generate(tasks):
    """Generator tasks of bench.py run in spawned processes (each object
    has its own random stream, so the parts equal the whole)."""
    import multiprocessing as mp
    import bench
    procs = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(bench._gen, tasks, chunksize=1)


def _box_candidates(mr, mS, tau):
    """Indices of the boxes of mS within tau (MINDIST) of box mr."""
    g = np.maximum(0, np.maximum(mS[:, :3] - mr[3:], mr[:3] - mS[:, 3:]))
    return np.nonzero(np.sqrt((g * g).sum(1)) <= tau * (1 + 1e-9))[0]


def _check_full_sets(res, R, S, tau, rl):
    """For each r in rl: the GPU's result set equals {s : d(r, s) <= tau}
    over every box candidate s, with the oracle's distances; distances
    reported exact match to 1e-12, brackets hold the oracle's value."""
    mR, mS = R.mbb().astype(np.float64), S.mbb().astype(np.float64)
    pr, ps = [], []
    for r in rl:
        for s in _box_candidates(mR[r], mS, tau):
            pr.append(r)
            ps.append(int(s))
    pr = np.array(pr, np.int32)
    ps = np.array(ps, np.int32)
    d = np.zeros(0)
    if len(pr):
        # the oracle on the objects involved only (the full sets' triangle
        # soups would be tens of GB)
        ur, us = np.unique(pr), np.unique(ps)
        d = oracle.pair_dists(subset(R, ur), subset(S, us), np.searchsorted(ur, pr).astype(np.int32),
                              np.searchsorted(us, ps).astype(np.int32))
    got = {}
    for a, b, lo, hi, dv, ex in zip(res.r.tolist(), res.s.tolist(), res.d_lo.tolist(), res.d_hi.tolist(),
                                    res.d.tolist(), res.exact.tolist()):
        got[(a, b)] = (lo, hi, dv, ex)
    hits = 0
    for a, b, w in zip(pr.tolist(), ps.tolist(), d.tolist()):
        if w <= tau:
            assert (a, b) in got, (a, b, w)
            lo, hi, dv, ex = got[(a, b)]
            assert lo <= w * (1 + 1e-12) + 1e-300 and w <= hi * (1 + 1e-12) + 1e-300
            if ex == 1:
                assert abs(dv - w) <= 1e-12 * w
            hits += 1
        else:
            assert (a, b) not in got, (a, b, w)
    extra = [p for p in got if p[0] in set(int(x) for x in rl) and p not in set(zip(pr.tolist(), ps.tolist()))]
    assert not extra, extra[:5]
    return hits


def test_knn50k_full_size_120_objects(ctx):
    """The k-NN workload at full size; the neighbour lists of 120 objects r
    equal the oracle's (ids bit-exact, order (d, s))."""
    from paper_2604_19982_gb300 import pj
    import test_gpu_knn as K
    w = configs.knn50k()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    res = ctx.join(gR, gS, pj.KNN, k=3, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST)
    assert res.n == 3 * w.R.n
    rl = np.sort(np.random.default_rng(5).choice(w.R.n, 120, replace=False))
    K.check_knn(res, w.R, w.S, 3, rlist=rl)
    gR.free()
    gS.free()


def test_tubes2k_full_size_whole_result_sets(ctx):
    """2,000 tubes x 200,000 blobs, side 2,320, tau = 2: the whole result
    sets of eight tubes (the six shortest, two at random) against the
    oracle's distances of all their box candidates."""
    from paper_2604_19982_gb300 import pj
    import bench
    parts = _generate(bench._parts("tubes", 2000, 2320.0, 0, 0, 32) + bench._parts("blobs", 200_000, 2320.0, 0, 1,
                                                                                    32))
    R, S = concat(parts[:32]), concat(parts[32:])
    gR, gS = ctx.load_set(R), ctx.load_set(S)
    res = ctx.join(gR, gS, pj.WITHIN, tau=2.0, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE)
    assert res.n > 0
    nf = np.diff(R.face_off[R.n_lods - 1])
    rl = np.concatenate([np.argsort(nf)[:6], np.random.default_rng(6).choice(R.n, 2, replace=False)])
    rl = np.unique(rl)
    hits = _check_full_sets(res, R, S, 2.0, rl)
    assert hits > 0
    gR.free()
    gS.free()


def test_stream2m_two_chunks_full_size(ctx):
    """Two of the 64 chunks of the streamed 2,000,000 blobs (chunks 0 and
    37, 31,250 blobs each) streamed against all 20,000 tubes, tau = 1: the
    whole result sets of sampled blobs of both chunks, and the streamed
    result equal to the resident join of the same chunks."""
    from paper_2604_19982_gb300 import pj
    import bench
    tasks = bench._parts("tubes", 20_000, 5000.0, 0, 1, 64) + [("chunk", 0, 0, 64), ("chunk", 37, 0, 64)]
    parts = _generate(tasks)
    S = concat(parts[:-2])
    chunks = parts[-2:]
    gS = ctx.load_set(S)
    gR = ctx.load_set_streamed(sum(c.n for c in chunks), 2, lambda c: chunks[c])
    fl = dict(prec=pj.FP32, flags=pj.TILE_PRUNE | pj.AUTOTUNE)
    res = ctx.join(gR, gS, pj.WITHIN, tau=1.0, **fl)
    both = concat(chunks)
    gB = ctx.load_set(both)
    ref = ctx.join(gB, gS, pj.WITHIN, tau=1.0, **fl)
    assert res.pairs() == ref.pairs() and np.array_equal(res.d_lo, ref.d_lo) and np.array_equal(res.d_hi, ref.d_hi)
    # sampled blobs of each chunk: four with results, four with candidates
    mB, mS = both.mbb().astype(np.float64), S.mbb().astype(np.float64)
    rng = np.random.default_rng(7)
    hit = np.unique(res.r)
    rl = []
    for lo, hi in ((0, chunks[0].n), (chunks[0].n, both.n)):
        h = hit[(hit >= lo) & (hit < hi)]
        rl += list(rng.choice(h, min(4, len(h)), replace=False))
        cand = [r for r in rng.permutation(np.arange(lo, hi))[:400] if len(_box_candidates(mB[r], mS, 1.0))]
        rl += cand[:4]
    rl = np.unique(np.array(rl, np.int64))
    sub_ids = rl
    Rs = subset(both, sub_ids)
    # the oracle on the sample, ids mapped back
    mask = np.isin(res.r, rl)

    class _Res:
        pass
    rr = _Res()
    remap = {int(g): i for i, g in enumerate(sub_ids)}
    rr.r = np.array([remap[int(x)] for x in res.r[mask]], np.int64)
    for f in ("s", "d_lo", "d_hi", "d", "exact"):
        setattr(rr, f, getattr(res, f)[mask])
    hits = _check_full_sets(rr, Rs, S, 1.0, np.arange(len(sub_ids)))
    assert hits >= 4
    gR.free()
    gB.free()
    gS.free()
