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
