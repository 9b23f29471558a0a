"""Pins of the CPU oracle against facts fixed by the paper and by geometry,
independent of the oracle's own code:

* closed forms (hand-derived dyadic distances, tests/golden)
* an optimality certificate for every triangle pair: the returned points lie
  on their triangles and the plane through them, normal to their difference,
  separates the triangles (for convex sets that proves the distance minimal)
* object level: axis-aligned boxes at a known gap, coincident and
  interpenetrating meshes, symmetry, bounding-box and anchor brackets
* joins: brute force over all pairs equals the pruned join; monotonicity in
  tau and k; facet-order permutation invariance; k-NN by full sort
* Eq. 1 / Eq. 2: every LoD bracket contains the full-resolution distance
* Algorithm 6 (corrected reading): the narrative of Fig. "Progressive
  Candidate Pruning for a k-NN Query" and soundness on random intervals
"""
import os

import numpy as np
import pytest

import oracle
from oracle import knn_prune
from synth import box_triangles, configs, from_triangles

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _closed_forms():
    out = []
    for line in open(os.path.join(GOLD, "tri_closed_forms.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lab, P, Q, d = [x.strip() for x in line.split("|")]
        out.append((lab, np.array(P.split(), float).reshape(3, 3), np.array(Q.split(), float).reshape(3, 3),
                    float(d)))
    return out


@pytest.mark.parametrize("case", _closed_forms(), ids=lambda c: c[0])
def test_tri_closed_forms(case):
    lab, P, Q, d = case
    got, cp = oracle.tri_dist(P[None], Q[None])
    assert got[0] == pytest.approx(d, abs=1e-15), lab
    got2, _ = oracle.tri_dist(Q[None], P[None])
    assert got2[0] == pytest.approx(d, abs=1e-15), lab
    assert np.linalg.norm(cp[0, 0] - cp[0, 1]) == pytest.approx(d, abs=1e-15)


def test_pierce_is_missed_by_the_fifteen_candidates():
    """The pierce fixture has distance 0, yet every vertex-to-triangle and
    edge-to-edge distance is positive (so the meeting test is necessary)."""
    case = [c for c in _closed_forms() if c[0] == "pierce"][0]
    _, P, Q, _ = case
    cands = []
    for i in range(3):
        cands.append(oracle.point_tri_dist(P[i], Q))
        cands.append(oracle.point_tri_dist(Q[i], P))
    # edge-edge distances via degenerate (segment) triangles
    for i in range(3):
        for j in range(3):
            sp = np.array([P[i], P[(i + 1) % 3], P[(i + 1) % 3]])
            sq = np.array([Q[j], Q[(j + 1) % 3], Q[(j + 1) % 3]])
            cands.append(oracle.tri_dist(sp[None], sq[None])[0][0])
    assert min(cands) > 0.4
    assert oracle.tri_dist(P[None], Q[None])[0][0] == 0.0


# ---------------------------------------------------------------- certificate


def _in_triangle(x, T, tol):
    """Is x in the convex hull of T's vertices (non-negative least squares)?"""
    from scipy.optimize import nnls
    A = np.vstack([T.T, np.ones((1, 3)) * 10.0])
    b = np.concatenate([x, [10.0]])
    _, res = nnls(A, b)
    return res <= tol


def _random_pairs(rng, n):
    P = rng.normal(size=(n, 3, 3))
    Q = rng.normal(size=(n, 3, 3)) + rng.normal(size=(n, 1, 3)) * rng.uniform(0, 3, size=(n, 1, 1))
    return P, Q


def _degenerate_pairs(rng):
    out = []
    for _ in range(300):
        P = rng.normal(size=(3, 3))
        kind = rng.integers(0, 8)
        Q = rng.normal(size=(3, 3))
        if kind == 0:      # shared vertex
            Q[0] = P[rng.integers(0, 3)]
        elif kind == 1:    # shared edge
            i = rng.integers(0, 3)
            Q[0], Q[1] = P[i], P[(i + 1) % 3]
        elif kind == 2:    # coplanar
            n = np.cross(P[1] - P[0], P[2] - P[0])
            n /= np.linalg.norm(n)
            Q = Q - ((Q - P[0]) @ n)[:, None] * n
        elif kind == 3:    # parallel edges
            Q[1] = Q[0] + (P[1] - P[0]) * rng.uniform(0.2, 2)
        elif kind == 4:    # sliver
            Q[2] = Q[0] + (Q[1] - Q[0]) * 0.5 + rng.normal(size=3) * 1e-7
        elif kind == 5:    # zero area (collinear)
            Q[2] = Q[0] + (Q[1] - Q[0]) * rng.uniform(-1, 2)
        elif kind == 6:    # point
            Q[1] = Q[0]
            Q[2] = Q[0]
        elif kind == 7:    # parallel planes, small gap
            n = np.cross(P[1] - P[0], P[2] - P[0])
            n /= np.linalg.norm(n)
            Q = Q - ((Q - P[0]) @ n)[:, None] * n + n * rng.uniform(1e-3, 0.5)
        out.append((P, Q))
    return np.array([p for p, _ in out]), np.array([q for _, q in out])


def _certify(P, Q, d, cp, tol=1e-9):
    """Check feasibility of the returned points and, for d above rounding
    level, that the plane through them normal to p - q separates P and Q."""
    bad = []
    for i in range(P.shape[0]):
        p, q = cp[i, 0], cp[i, 1]
        scale = max(1.0, np.abs(P[i]).max(), np.abs(Q[i]).max())
        if abs(np.linalg.norm(p - q) - d[i]) > tol * scale:
            bad.append((i, "dist"))
            continue
        if not _in_triangle(p, P[i], tol * scale) or not _in_triangle(q, Q[i], tol * scale):
            bad.append((i, "feasible"))
            continue
        if d[i] > 1e-13 * scale:
            w = (p - q) / d[i]
            if (P[i] @ w).min() < w @ p - tol * scale or (Q[i] @ w).max() > w @ q + tol * scale:
                bad.append((i, "separation"))
    return bad


def test_tri_certificate_random():
    rng = np.random.default_rng(7)
    P, Q = _random_pairs(rng, 4000)
    d, cp = oracle.tri_dist(P, Q)
    assert (d >= 0).all()
    assert (d == 0).sum() > 50 and (d > 0).sum() > 1000   # both regimes exercised
    assert _certify(P, Q, d, cp) == []


def test_tri_certificate_degenerate():
    rng = np.random.default_rng(11)
    P, Q = _degenerate_pairs(rng)
    d, cp = oracle.tri_dist(P, Q)
    assert _certify(P, Q, d, cp, tol=1e-8) == []


def test_certificate_catches_planted_mistake():
    """A closest-point pair shifted off the optimum fails the certificate."""
    rng = np.random.default_rng(3)
    P, Q = _random_pairs(rng, 200)
    d, cp = oracle.tri_dist(P, Q)
    keep = d > 0.1
    cp2 = cp.copy()
    cp2[:, 0] = (cp[:, 0] + P[:, 0]) / 2.0   # a feasible but wrong point on P
    d2 = np.linalg.norm(cp2[:, 0] - cp2[:, 1], axis=1)
    moved = keep & (np.linalg.norm(cp2[:, 0] - cp[:, 0], axis=1) > 1e-3)
    bad = _certify(P[moved], Q[moved], d2[moved], cp2[moved])
    assert len(bad) == moved.sum()


# ---------------------------------------------------------------- objects


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("gap", [0.125, 0.5, 3.0])
def test_boxes_at_known_gap(axis, gap):
    lo = np.zeros(3)
    A = box_triangles(lo, lo + 1.0)
    off = np.array([0.25, -0.5, 0.125])
    off[axis] = 1.0 + gap
    B = box_triangles(off, off + 1.0)
    assert oracle.obj_dist(A, B) == gap          # exact: dyadic arithmetic


def test_boxes_diagonal_gap():
    A = box_triangles(np.zeros(3), np.ones(3))
    o = np.array([1.375, 1.5, 0.25])               # gaps 3/8, 1/2 -> 5/8
    B = box_triangles(o, o + 1.0)
    assert oracle.obj_dist(A, B) == 0.625


def test_coincident_and_interpenetrating_meshes(blobs100):
    R = blobs100.R
    T = R.triangles(R.n_lods - 1, 0)
    assert oracle.obj_dist(T, T) == 0.0
    shifted = T + np.float32(0.05)
    assert oracle.obj_dist(T, shifted) == 0.0


def test_object_brackets_and_symmetry(blobs100):
    R, S = blobs100.R, blobs100.S
    rng = np.random.default_rng(5)
    pr = rng.integers(0, R.n, 60).astype(np.int32)
    ps = rng.integers(0, S.n, 60).astype(np.int32)
    d = oracle.pair_dists(R, S, pr, ps)
    d_t = oracle.pair_dists(S, R, ps, pr)
    assert np.allclose(d, d_t, rtol=1e-12, atol=1e-12)
    assert (d >= 0).all()
    mR, mS = R.mbb().astype(np.float64), S.mbb().astype(np.float64)
    gap = np.maximum(0, np.maximum(mS[ps, :3] - mR[pr, 3:], mR[pr, :3] - mS[ps, 3:]))
    mind = np.sqrt((gap ** 2).sum(1))
    anc = np.linalg.norm(R.anchor[pr].astype(np.float64) - S.anchor[ps], axis=1)
    assert (mind <= d * (1 + 1e-12) + 1e-12).all()
    assert (d <= anc * (1 + 1e-12) + 1e-12).all()


def test_facet_permutation_invariance(blobs100):
    R, S = blobs100.R, blobs100.S
    A = R.triangles(R.n_lods - 1, 3)
    B = S.triangles(S.n_lods - 1, 7)
    rng = np.random.default_rng(1)
    d0 = oracle.obj_dist(A, B)
    d1 = oracle.obj_dist(A[rng.permutation(len(A))], B[rng.permutation(len(B))])
    assert d0 == d1


# ---------------------------------------------------------------- joins


def test_within_pruned_equals_brute(blobs100):
    R, S = blobs100.R, blobs100.S
    rl = np.arange(0, 100, 12)
    a = oracle.join_within(R, S, 0.5, prune=True, rlist=rl)
    b = oracle.join_within(R, S, 0.5, prune=False, rlist=rl)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert len(a[0]) > 0


def test_within_pruned_equals_brute_on_touching_boxes():
    """Boxes and tetrahedra touching exactly (face, edge, vertex contacts,
    one-step gaps and overlaps): many S boxes start exactly where an R box
    ends, the boundary case of the box sweep; the pruned join must still
    equal brute force over all pairs, for tau = 0 and one step above."""
    from meet_cases import contact_sets
    for seed in (0, 1):
        R, S = contact_sets(seed)
        for tau in (0.0, 1e-3):
            a = oracle.join_within(R, S, tau, prune=True)
            b = oracle.join_within(R, S, tau, prune=False)
            for x, y in zip(a, b):
                assert np.array_equal(x, y), (seed, tau)
            if tau == 0.0:   # the designed contacts: both outcomes in numbers
                own = {(i, i) for i in range(R.n)}
                assert 60 < len(own & set(zip(a[0].tolist(), a[1].tolist()))) < R.n - 40


def test_within_monotone_in_tau(blobs100):
    R, S = blobs100.R, blobs100.S
    prev = set()
    for tau in (0.0, 0.25, 0.5, 1.0):
        r, s, d = oracle.join_within(R, S, tau)
        cur = set(zip(r.tolist(), s.tolist()))
        assert prev <= cur
        assert (d <= tau).all()
        prev = cur
    r0, s0, d0 = oracle.join_within(R, S, 0.0)
    assert (d0 == 0).all() and len(r0) > 0      # intersection join is tau = 0


def test_within_symmetry(blobs100):
    R, S = blobs100.R, blobs100.S
    r, s, d = oracle.join_within(R, S, 0.5)
    r2, s2, d2 = oracle.join_within(S, R, 0.5)
    a = sorted(zip(r.tolist(), s.tolist()))
    b = sorted(zip(s2.tolist(), r2.tolist()))
    assert a == b


def test_knn_by_full_sort_and_nesting(blobs100):
    R, S = blobs100.R, blobs100.S
    rl = np.array([0, 17, 42, 99])
    r3, s3, d3 = oracle.join_knn(R, S, 3, rlist=rl)
    r4, s4, d4 = oracle.join_knn(R, S, 4, rlist=rl)
    pr = np.repeat(rl, S.n).astype(np.int32)
    ps = np.tile(np.arange(S.n), len(rl)).astype(np.int32)
    dall = oracle.pair_dists(R, S, pr, ps).reshape(len(rl), S.n)
    for i, r in enumerate(rl):
        order = sorted(range(S.n), key=lambda s: (dall[i, s], s))
        assert s3[r3 == r].tolist() == order[:3]
        assert s4[r4 == r].tolist() == order[:4]
        assert np.array_equal(d3[r3 == r], dall[i, order[:3]])


def test_knn_fewer_objects_than_k(blobs100):
    R, S = blobs100.R, blobs100.S
    small = from_triangles([S.triangles(S.n_lods - 1, i) for i in range(2)])
    r, s, d = oracle.join_knn(R, small, 5, rlist=np.array([0, 1]))
    assert len(r) == 4 and set(s.tolist()) == {0, 1}


# ---------------------------------------------------------------- Eq. 1 / 2


def test_lod_bounds_bracket_distance(blobs100):
    R, S = blobs100.R, blobs100.S
    r, s, _ = oracle.join_within(R, S, 2.0)
    rng = np.random.default_rng(2)
    pick = rng.choice(len(r), size=min(40, len(r)), replace=False)
    pr, ps = r[pick], s[pick]
    d = oracle.pair_dists(R, S, pr, ps)
    lb, ub = oracle.pair_bounds(R, S, pr, ps, lod=0)
    assert (lb <= d).all() and (d <= ub).all()
    assert (ub - lb > 0).all()
    lbF, ubF = oracle.pair_bounds(R, S, pr, ps, lod=R.n_lods - 1)
    assert np.array_equal(lbF, d) and np.array_equal(ubF, d)


def test_lod_bounds_catch_dropped_hausdorff_term(blobs100):
    """Planting a mistake (ph ignored) breaks the Eq. 2 bracket somewhere."""
    R, S = blobs100.R, blobs100.S
    r, s, _ = oracle.join_within(R, S, 1.0)
    d = oracle.pair_dists(R, S, r, s)
    broken = 0
    for i in range(len(r)):
        A = R.triangles(0, r[i])
        B = S.triangles(0, s[i])
        z = np.zeros(len(A), np.float32)
        zb = np.zeros(len(B), np.float32)
        lb, _ = oracle.lod_bounds(A, R.hd_of(0, r[i]), z, B, S.hd_of(0, s[i]), zb)
        broken += lb > d[i]
    assert broken > 0


def _tiny_blob():
    return configs.blob_set(1, 10.0, 3, 0, subs=(1, 2))


def test_hausdorff_bounds_by_sampling():
    """hd: points sampled on coarse facets stay within hd of the fine mesh;
    ph: fine points lie within ph(f') of some coarse facet f'."""
    B = _tiny_blob()
    coarse = B.triangles(0, 0).astype(np.float64)
    fine = B.triangles(1, 0)
    hd = B.hd_of(0, 0).astype(np.float64)
    ph = B.ph_of(0, 0).astype(np.float64)
    g = np.array([(a, b) for a in np.linspace(0, 1, 6) for b in np.linspace(0, 1, 6) if a + b <= 1])
    for f in range(0, coarse.shape[0], 3):
        T = coarse[f]
        pts = T[0] + g[:, :1] * (T[1] - T[0]) + g[:, 1:] * (T[2] - T[0])
        for p in pts:
            assert oracle.point_mesh_dist(p, fine) <= hd[f] + 1e-9
    fv = fine.reshape(-1, 3).astype(np.float64)
    for p in fv[::7]:
        gaps = [oracle.point_tri_dist(p, coarse[f]) - ph[f] for f in range(coarse.shape[0])]
        assert min(gaps) <= 1e-9


def test_tube_hausdorff_by_sampling():
    T = configs.tube_set(1, 50.0, 4, 0)
    for lod in (0, 1):
        coarse = T.triangles(lod, 0).astype(np.float64)
        fine = T.triangles(T.n_lods - 1, 0)
        hd = T.hd_of(lod, 0).astype(np.float64)
        rng = np.random.default_rng(lod)
        for f in rng.choice(coarse.shape[0], 25, replace=False):
            tri = coarse[f]
            for a, b in ((1 / 3, 1 / 3), (0.1, 0.8), (0.8, 0.1), (0.5, 0.0)):
                p = tri[0] + a * (tri[1] - tri[0]) + b * (tri[2] - tri[0])
                assert oracle.point_mesh_dist(p, fine) <= hd[f] + 1e-9


def _ph_gap(p, coarse, ph, near=None):
    """min over coarse facets f of (distance(p, f) - ph[f]); with `near`,
    over the `near` facets with the closest centroids only."""
    fs = range(coarse.shape[0])
    if near is not None:
        c = coarse.mean(axis=1)
        fs = np.argsort(((c - p) ** 2).sum(1))[:near]
    return min(oracle.point_tri_dist(p, coarse[f]) - ph[f] for f in fs)


def test_tube_ph_by_sampling():
    """ph: every point of the original tube surface lies within ph(f') of
    some coarse facet f' (the Eq. 2 direction), checked on fine vertices
    and on points inside fine facets, against the coarse facets nearest to
    each point (the facet whose patch holds the point is among them)."""
    T = configs.tube_set(1, 50.0, 4, 0)
    fine = T.triangles(T.n_lods - 1, 0).astype(np.float64)
    rng = np.random.default_rng(7)
    pick = rng.choice(fine.shape[0], 80, replace=False)
    w = rng.dirichlet((1.0, 1.0, 1.0), size=80)
    pts = np.vstack([fine.reshape(-1, 3)[::17], np.einsum("ij,ijk->ik", w, fine[pick])])
    for lod in (0, 1):
        coarse = T.triangles(lod, 0).astype(np.float64)
        ph = T.ph_of(lod, 0).astype(np.float64)
        for p in pts:
            assert _ph_gap(p, coarse, ph, near=12) <= 1e-9, (lod, p)


def test_tube_ph_catches_a_shrunk_bound():
    """The same check over all coarse facets fails once ph is halved (the
    pin is not vacuous)."""
    T = configs.tube_set(1, 50.0, 4, 0)
    fine = T.triangles(T.n_lods - 1, 0).astype(np.float64).reshape(-1, 3)
    coarse = T.triangles(0, 0).astype(np.float64)
    ph = T.ph_of(0, 0).astype(np.float64) * 0.5
    pts = fine[np.random.default_rng(8).choice(fine.shape[0], 30, replace=False)]
    assert sum(_ph_gap(p, coarse, ph) > 1e-9 for p in pts) > 0


# ---------------------------------------------------------------- Alg 6


def _fig_stages():
    rows = []
    for line in open(os.path.join(GOLD, "knn_fig_bounds.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        stage, vals, exp = [x.strip() for x in line.split("|")]
        v = np.array(vals.split(), float).reshape(-1, 3)
        rows.append((stage, v[:, 0].astype(int).tolist(), v[:, 1].tolist(), v[:, 2].tolist(), exp.split()))
    return rows


def test_knn_prune_figure_narrative():
    code = {"U": knn_prune.UNDECIDED, "C": knn_prune.CONFIRMED, "R": knn_prune.REMOVED}
    status = [knn_prune.UNDECIDED] * 4
    for stage, ids, lb, ub, exp in _fig_stages():
        status = knn_prune.prune_round(2, ids, lb, ub, status)
        assert status == [code[e] for e in exp], stage


def test_knn_prune_sound_on_random_intervals():
    rng = np.random.default_rng(9)
    for trial in range(400):
        n = int(rng.integers(1, 9))
        k = int(rng.integers(1, 5))
        d = rng.integers(0, 6, size=n).astype(float)       # many exact ties
        ids = list(range(n))
        truth = set(sorted(ids, key=lambda i: (d[i], i))[:k])
        status = [knn_prune.UNDECIDED] * n
        for width in (3.0, 1.5, 0.5, 0.0):
            lb = (d - rng.uniform(0, width, n)).tolist()
            ub = (d + rng.uniform(0, width, n)).tolist()
            status = knn_prune.prune_round(k, ids, lb, ub, status)
            for i in ids:
                if status[i] == knn_prune.CONFIRMED:
                    assert i in truth
                if status[i] == knn_prune.REMOVED:
                    assert i not in truth
        assert all(s != knn_prune.UNDECIDED for s in status)   # exact bounds resolve all
