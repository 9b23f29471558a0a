"""Per-LoD Eq. 1 / Eq. 2 bounds of object pairs (pj_pair_bounds, every facet
pair evaluated) against the oracle's bounds."""
import numpy as np
import pytest

import oracle
from synth import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2604_19982_gb300 import pj
    w = configs.blobs100()
    ctx = pj.Context(0)
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    r, s, _ = oracle.join_within(w.R, w.S, 1.5)
    rng = np.random.default_rng(4)
    pick = np.sort(rng.choice(len(r), min(60, len(r)), replace=False))
    yield w, ctx, gR, gS, r[pick], s[pick]
    ctx.close()


@pytest.mark.parametrize("lod", [0, 1])
def test_fp64_bounds_match_oracle(setup, lod):
    from paper_2604_19982_gb300 import pj
    w, ctx, gR, gS, pr, ps = setup
    lb, ub = ctx.pair_bounds(gR, gS, pr, ps, lod, pj.FP64)
    olb, oub = oracle.pair_bounds(w.R, w.S, pr, ps, lod)
    olb = np.maximum(olb, 0.0)
    assert (np.abs(ub - oub) <= 1e-12 * oub + 1e-14).all()
    assert (np.abs(lb - olb) <= 1e-12 * np.abs(olb) + 1e-14).all()
    if lod == w.R.n_lods - 1:
        assert np.array_equal(lb, ub)


@pytest.mark.parametrize("lod", [0, 1])
def test_fp32_bounds_bracket_oracle(setup, lod):
    from paper_2604_19982_gb300 import pj
    w, ctx, gR, gS, pr, ps = setup
    lb, ub = ctx.pair_bounds(gR, gS, pr, ps, lod, pj.FP32)
    olb, oub = oracle.pair_bounds(w.R, w.S, pr, ps, lod)
    olb = np.maximum(olb, 0.0)
    assert (lb <= olb).all() and (oub <= ub).all()
    # the bracket widens by the per-tile forward error bound, dominated by
    # 8 sqrt(u) L with L the longest edge (~1.4 at the coarsest blob LoD)
    tol = 5e-3 if lod == 0 else 2e-3
    assert (ub - oub < tol).all() and (olb - lb < tol).all()


def test_bounds_bracket_full_resolution_distance(setup):
    from paper_2604_19982_gb300 import pj
    w, ctx, gR, gS, pr, ps = setup
    d = oracle.pair_dists(w.R, w.S, pr, ps)
    for prec in (pj.FP64, pj.FP32):
        lb, ub = ctx.pair_bounds(gR, gS, pr, ps, 0, prec)
        assert (lb <= d * (1 + 1e-12)).all() and (d <= ub * (1 + 1e-12)).all()


def _single_facet_sets(P, Q):
    """One object per triangle, two LoDs: LoD 0 is the same triangle with
    hd = ph = 0 (so the coarse-LoD single-precision path computes plain
    distances), LoD 1 the original."""
    from synth import from_triangles
    return from_triangles([p[None] for p in P], n_lods=2), from_triangles([q[None] for q in Q], n_lods=2)


@pytest.mark.parametrize("kind", ["random", "near_parallel", "piercing"])
def test_fp32_coarse_path_within_its_margin(kind):
    """The coarse-LoD single-precision test (square root by
    sqrt.approx.ftz, segment parameters by the fast reciprocal) directly:
    each pair's [lb, ub] from the coarse step brackets the oracle's
    distance (hd = ph = 0, so lb = d32 - eps and ub = d32 + eps); the
    bracket is narrow where the conditioning is good."""
    from paper_2604_19982_gb300 import pj
    import test_gpu_tri as T
    rng = np.random.default_rng({"random": 51, "near_parallel": 52, "piercing": 53}[kind])
    n = 6000
    P, Q = {"random": T.random_pairs, "near_parallel": T.near_parallel_pairs,
            "piercing": T.piercing_pairs}[kind](rng, n)
    R, S = _single_facet_sets(P, Q)
    ref, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    ctx = pj.Context(0)
    try:
        gR, gS = ctx.load_set(R), ctx.load_set(S)
        idx = np.arange(n, dtype=np.int32)
        lb, ub = ctx.pair_bounds(gR, gS, idx, idx, 0, pj.FP32)
        assert (lb <= ref).all() and (ref <= ub).all()
        L = np.linalg.norm(P[:, 1].astype(np.float64) - P[:, 0], axis=1)
        if kind == "random":
            assert np.median(ub - lb) < 2e-2 * np.median(L)
    finally:
        ctx.close()
