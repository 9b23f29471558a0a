"""Pins of the voxel oracle (oracle/voxel.py): k-means on a planted case and
its update rule, the voxel partition's defining properties, the voxel-pair
bounds against brute-force facet distances, and the voxel-pair pruning of
Algorithm 2 against the pair that realises the distance.  CPU only."""
import numpy as np
import pytest

import oracle
from oracle import voxel as vx
from synth import configs
from voxel_cases import empty_and_two_triangles


def _object_tris(ms, o):
    """Triangles [F_l, 9] of object o at every LoD (coarsest first)."""
    out = []
    for lod in range(ms.n_lods):
        tri, off, _, _ = oracle.soup(ms, lod)
        out.append(tri[off[o]:off[o + 1]].astype(np.float64))
    return out


def _coarse_verts(ms, o):
    """Vertex array [V, 3] of object o at the coarsest LoD."""
    vo = ms.vert_off[0]
    return ms.verts[0][vo[o]:vo[o + 1]].astype(np.float64)


def _vox(ms, o):
    return vx.voxelize(_object_tris(ms, o), _coarse_verts(ms, o))


def test_voxel_count_rule():
    assert vx.voxel_count(1280, 80) == 26       # round(25.6)
    assert vx.voxel_count(100, 50) == 2
    assert vx.voxel_count(10, 4) == 1           # at least one
    assert vx.voxel_count(50_000, 12) == 12     # at most the coarsest LoD's facets
    # round-half-up of F / 50 in integers: (F + 25) // 50 for every F up to 10^6
    F = np.arange(0, 1_000_001)
    k = np.floor(vx.VOXEL_FRACTION * F + 0.5).astype(np.int64)
    assert np.array_equal(k, (F + 25) // 50)


def test_initial_centres_evenly_spaced():
    v = np.arange(30, dtype=np.float64).reshape(10, 3)
    # floor(0.5 * 10 / 3) = 1, floor(1.5 * 10 / 3) = 5, floor(2.5 * 10 / 3) = 8
    assert np.array_equal(vx.initial_centres(v, 3), v[[1, 5, 8]])
    assert np.array_equal(vx.initial_centres(v, 10), v)
    assert np.array_equal(vx.initial_centres(v, 1), v[[5]])


def test_centroid_and_squares_fixed_order():
    t = np.array([[0.1, 0.2, 0.3, 1e16, 1.0, 2.0, -1e16, 3.0, 5.0]])
    # (v0 + v1) + v2 loses v0.x to rounding against 1e16
    assert vx.centroids(t)[0, 0] == ((0.1 + 1e16) + -1e16) / 3.0
    d = np.array([1e8, 1.0, 1e-8])
    assert vx.sq3(d) == (1e8 * 1e8 + 1.0 * 1.0) + 1e-8 * 1e-8


def test_kmeans_recovers_two_planted_clusters():
    # two tight clusters far apart, centres started inside each: after the
    # updates every centre is its cluster's mean (closed form)
    rng = np.random.default_rng(0)
    a = rng.normal(0.0, 0.1, (40, 3))
    b = rng.normal(0.0, 0.1, (25, 3)) + [50.0, -20.0, 7.0]
    cent = np.concatenate([b, a])
    c = vx.kmeans(cent, np.array([a[3], b[5]]))
    assert np.allclose(c[0], a.mean(axis=0), atol=1e-12)
    assert np.allclose(c[1], b.mean(axis=0), atol=1e-12)
    lab = vx.assign(cent, c)
    assert (lab[:25] == 1).all() and (lab[25:] == 0).all()


def test_kmeans_one_update_by_brute_force():
    # one update: each centre is the mean of the centroids nearer to it than
    # to any other centre (checked by explicit loops), an empty one stays
    rng = np.random.default_rng(1)
    cent = rng.uniform(-5, 5, (60, 3))
    init = np.array([[0.0, 0.0, 0.0], [4.0, 4.0, 4.0], [-4.0, 3.0, 0.0], [100.0, 100.0, 100.0]])
    c = vx.kmeans(cent, init, updates=1)
    sums = [np.zeros(3) for _ in init]
    counts = [0] * len(init)
    for p in cent:
        best, bj = None, -1
        for j, q in enumerate(init):
            d = float(np.dot(p - q, p - q))
            if best is None or d < best:
                best, bj = d, j
        sums[bj] = sums[bj] + p
        counts[bj] += 1
    for j in range(len(init)):
        want = sums[j] / counts[j] if counts[j] else init[j]
        assert np.allclose(c[j], want, atol=1e-12)
    assert counts[3] == 0 and np.array_equal(c[3], init[3])


@pytest.mark.parametrize("kind", ["blob", "tube"])
def test_voxelize_partition_properties(kind):
    ms = configs.blob_set(3, 40.0, 2, 0) if kind == "blob" else \
        configs.tube_set(2, 200.0, 2, 1, length_range=(50.0, 70.0))
    for o in range(ms.n):
        tris = _object_tris(ms, o)
        v = vx.voxelize(tris, _coarse_verts(ms, o))
        k = v["centres"].shape[0]
        assert k == vx.voxel_count(tris[-1].shape[0], tris[0].shape[0])
        for t, lab in zip(tris, v["labels"]):
            assert lab.shape[0] == t.shape[0] and lab.min() >= 0 and lab.max() < k
            # every facet's voxel is the one whose centre is nearest to its centroid
            cen = t.reshape(-1, 3, 3).mean(axis=1)
            d2 = ((cen[:, None, :] - v["centres"][None]) ** 2).sum(2)
            assert (d2[np.arange(len(lab)), lab] <= d2.min(axis=1)).all()
        pts = tris[-1].reshape(-1, 3, 3)
        for j in range(k):
            members = pts[v["labels"][-1] == j].reshape(-1, 3)
            if members.shape[0] == 0:
                assert np.isinf(v["boxes"][j]).all()
                continue
            # the box holds the members and touches them on every side
            assert (members >= v["boxes"][j, :3]).all() and (members <= v["boxes"][j, 3:]).all()
            assert np.allclose(members.min(0), v["boxes"][j, :3]) and np.allclose(members.max(0), v["boxes"][j, 3:])
            # the anchor is a member vertex, none nearer to the box centre
            a = v["anchors"][j]
            assert (np.abs(members - a).sum(1) == 0).any()
            c = 0.5 * (v["boxes"][j, :3] + v["boxes"][j, 3:])
            assert np.dot(a - c, a - c) <= ((members - c) ** 2).sum(1).min() + 1e-12


def _pairs():
    # a blob against a short tube, and two blobs, placed close together
    R = configs.blob_set(2, 12.0, 3, 0)
    S = configs.tube_set(1, 60.0, 3, 1, length_range=(50.0, 55.0))
    return [(R, 0, S, 0), (R, 0, R, 1)]


def test_voxel_pair_bounds_bracket_facet_distances():
    for Rm, r, Sm, s in _pairs():
        tr, ts = _object_tris(Rm, r), _object_tris(Sm, s)
        vr, vs = _vox(Rm, r), _vox(Sm, s)
        lb, ub, op_lb, op_ub = vx.voxel_pair_bounds(vr, vs)
        A = tr[-1].reshape(-1, 3, 3)
        B = ts[-1].reshape(-1, 3, 3)
        d = oracle.obj_dist(A, B)
        assert op_lb <= d * (1 + 1e-12) + 1e-12 and d <= op_ub * (1 + 1e-12) + 1e-12
        la, lb_ = vr["labels"][-1], vs["labels"][-1]
        rng = np.random.default_rng(4)
        pairs = [(i, j) for i in range(lb.shape[0]) for j in range(lb.shape[1]) if np.isfinite(lb[i, j])]
        for i, j in [pairs[q] for q in rng.choice(len(pairs), min(12, len(pairs)), replace=False)]:
            dv = oracle.obj_dist(A[la == i], B[lb_ == j])
            assert lb[i, j] <= dv * (1 + 1e-12) + 1e-12 <= ub[i, j] * (1 + 1e-12) + 2e-12


def test_pruning_keeps_the_voxel_pair_that_realises_the_distance():
    for Rm, r, Sm, s in _pairs():
        tr, ts = _object_tris(Rm, r), _object_tris(Sm, s)
        vr, vs = _vox(Rm, r), _vox(Sm, s)
        lb, ub, op_lb, op_ub = vx.voxel_pair_bounds(vr, vs)
        kept = vx.prune_voxel_pairs(lb, op_ub)
        # Algorithm 2 keeps exactly lb <= ub_o, in (i, j) order
        want = [(i, j) for i in range(lb.shape[0]) for j in range(lb.shape[1]) if lb[i, j] <= op_ub]
        assert [tuple(x) for x in kept.tolist()] == want
        assert 0 < len(want) < lb.size     # something kept, something pruned
        # the closest facet pair (brute force) lies in a kept voxel pair
        A = tr[-1].reshape(-1, 3, 3)
        B = ts[-1].reshape(-1, 3, 3)
        ia = np.repeat(np.arange(len(A)), len(B))
        ib = np.tile(np.arange(len(B)), len(A))
        dd, _ = oracle.tri_dist(A[ia], B[ib])
        best = int(np.argmin(dd))
        hold = (int(vr["labels"][-1][ia[best]]), int(vs["labels"][-1][ib[best]]))
        assert hold in want


def test_planted_mistake_box_centres_break_the_lower_bound():
    # a plausible slip -- the distance of the box centres instead of the
    # boxes' MINDIST -- overshoots the facet distance of some voxel pair, so
    # the bracket pin above would catch it
    Rm, r, Sm, s = _pairs()[0]
    tr, ts = _object_tris(Rm, r), _object_tris(Sm, s)
    vr, vs = _vox(Rm, r), _vox(Sm, s)
    A = tr[-1].reshape(-1, 3, 3)
    B = ts[-1].reshape(-1, 3, 3)
    broken = 0
    for i in range(vr["boxes"].shape[0]):
        for j in range(vs["boxes"].shape[0]):
            if not (np.isfinite(vr["boxes"][i, 0]) and np.isfinite(vs["boxes"][j, 0])):
                continue
            ci = 0.5 * (vr["boxes"][i, :3] + vr["boxes"][i, 3:])
            cj = 0.5 * (vs["boxes"][j, :3] + vs["boxes"][j, 3:])
            dv = oracle.obj_dist(A[vr["labels"][-1] == i], B[vs["labels"][-1] == j])
            broken += np.linalg.norm(ci - cj) > dv * (1 + 1e-9)
            if broken:
                return
    assert broken


def test_object_pruning_agrees_with_the_join():
    # pairs the voxel bounds decide are decided the same way by the exact join
    R = configs.blob_set(6, 14.0, 5, 0)
    S = configs.blob_set(6, 14.0, 5, 1)
    tau = 1.0
    r_, s_, _ = oracle.join_within(R, S, tau)
    res = set(zip(r_.tolist(), s_.tolist()))
    seen = [0, 0, 0]
    for r in range(R.n):
        vr = _vox(R, r)
        for s in range(S.n):
            vs = _vox(S, s)
            _, _, op_lb, op_ub = vx.voxel_pair_bounds(vr, vs)
            dec = vx.decide_within(op_lb, op_ub, tau)
            seen[dec] += 1
            if dec == 1:
                assert (r, s) in res
            elif dec == 2:
                assert (r, s) not in res
    assert seen[2] > 0


def test_set_helpers_match_the_per_object_calls():
    R = configs.blob_set(3, 12.0, 3, 0)
    S = configs.tube_set(2, 60.0, 3, 1, length_range=(50.0, 55.0))
    vR, vS = vx.voxelize_set(R), vx.voxelize_set(S)
    for o in range(R.n):
        a, b = vR[o], _vox(R, o)
        assert np.array_equal(a["centres"], b["centres"]) and np.array_equal(a["boxes"], b["boxes"])
        assert all(np.array_equal(x, y) for x, y in zip(a["labels"], b["labels"]))
    pr = np.array([0, 1, 2, 2])
    ps = np.array([0, 1, 0, 1])
    for tau in (-1.0, 1.0, 1e9):
        f = vx.voxel_filter(vR, vS, pr, ps, tau)
        for p in range(len(pr)):
            lb, ub, olb, oub = vx.voxel_pair_bounds(vR[pr[p]], vS[ps[p]])
            assert f["op_lb"][p] == olb and f["op_ub"][p] == oub
            assert np.array_equal(f["vp_lb"][f["vp_off"][p]:f["vp_off"][p + 1]], lb.reshape(-1))
            kept = f["kept"][f["kept_off"][p]:f["kept_off"][p + 1]]
            if f["status"][p] == 0:
                assert np.array_equal(kept, vx.prune_voxel_pairs(lb, oub))
            else:
                assert kept.shape[0] == 0
        if tau < 0:
            assert (f["status"] == 0).all()
        if tau == 1e9:
            assert (f["status"] == 1).all() and f["kept"].shape[0] == 0


def test_object_without_facets_has_no_voxels():
    ms = empty_and_two_triangles()
    vs = vx.voxelize_set(ms)
    assert vx.voxel_count(0, 0) == 0 and vs[0]["centres"].shape == (0, 3)
    assert all(lab.shape == (0,) for lab in vs[0]["labels"])
    assert vs[1]["centres"].shape == (1, 3)     # round(2 / 50) = 0, at least one
    f = vx.voxel_filter(vs, vs, np.array([0, 1]), np.array([1, 1]), 0.5)
    assert f["op_lb"][0] == np.inf and f["status"][0] == 2 and f["vp_off"][1] == 0
    assert f["op_lb"][1] == 0.0 and f["status"][1] == 1
    f = vx.voxel_filter(vs, vs, np.array([0]), np.array([0]), -1.0)
    assert f["status"][0] == 0 and f["kept"].shape == (0, 2)
