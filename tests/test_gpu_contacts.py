"""Intersection joins (tau = 0) of meshes that touch exactly or miss by one
float32 step, through the C ABI against the oracle.

Objects are boxes and tetrahedra with float32 (dyadic) coordinates: face
on face, edge on edge, vertex on vertex, a vertex of one on a face or edge
of the other, one-step gaps and one-step overlaps.  Intersection is d = 0
(section 3), and d = 0 exactly when two facets meet (section 2.1), so the
result sets must equal the oracle's pair for pair in every precision mode.
"""
import numpy as np
import pytest

import oracle
from meet_cases import contact_sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


MODES = {
    "fp64": dict(prec=0, flags=0),
    "fp32": dict(prec=1, flags=0),
    "fp32_prune": dict(prec=1, flags=16),
    "fp32_prune_exact": dict(prec=1, flags=16 | 1),
}


@pytest.mark.parametrize("seed", [0, 1])
@pytest.mark.parametrize("mode", list(MODES))
def test_touching_meshes_intersection(ctx, seed, mode):
    from paper_2604_19982_gb300 import pj
    R, S = contact_sets(seed)
    r, s, d = oracle.join_within(R, S, 0.0)
    want = list(zip(r.tolist(), s.tolist()))
    # the designed contacts: both outcomes present in numbers
    own = {(i, i) for i in range(R.n)}
    assert 60 < len(own & set(want)) < R.n - 40
    gR, gS = ctx.load_set(R), ctx.load_set(S)
    res = ctx.join(gR, gS, pj.INTERSECT, **MODES[mode])
    assert res.pairs() == want
    assert (res.d_lo == 0).all() and (res.d_hi == 0).all()
    # within a tau of one step: the near misses join, the overlaps stay
    res2 = ctx.join(gR, gS, pj.WITHIN, tau=1e-3, **MODES[mode])
    r2, s2, _ = oracle.join_within(R, S, 1e-3)
    assert res2.pairs() == list(zip(r2.tolist(), s2.tolist()))
    gR.free()
    gS.free()
