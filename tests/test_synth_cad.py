"""The CAD-like workload generator (synth/cad.py, stand-in for the paper's
ModelNet sets): closed parts, exact box coordinates, Hausdorff bounds by
sampling, replicas as exact translates, chunks equal to the whole set, and
oracle distances on hand-placed replicas.  CPU only."""
import numpy as np
import pytest

import oracle
from synth import cad, configs


def _edges_twice(F):
    e = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    return (cnt == 2).all()


@pytest.mark.parametrize("n", cad.BOX_GRID)
def test_box_parts_are_closed_and_exact(n):
    V, F = cad.box_mesh((1.0, 2.0, 3.0), (5.25, 2.5, 9.0), n)
    assert _edges_twice(F)
    assert F.shape[0] == 12 * n * n
    assert np.array_equal(V.astype(np.float32).astype(np.float64), V)
    # every vertex on the box surface
    on = np.isclose(V, [1.0, 2.0, 3.0], rtol=0, atol=0) | np.isclose(V, [5.25, 2.5, 9.0], rtol=0, atol=0)
    assert on.any(axis=1).all()


@pytest.mark.parametrize("m", cad.CYL_SEGMENTS)
def test_cylinder_parts_are_closed(m):
    V, F = cad.cylinder_mesh(3.0, -2.0, 0.5, 13.0, 1.5, m)
    assert _edges_twice(F)
    h = int(np.ceil(12.5 / cad.RING_SPACING))
    assert F.shape[0] == 2 * m * h + 2 * m
    r = np.hypot(V[:, 0] - 3.0, V[:, 1] + 2.0)
    assert np.allclose(r[:-2], 1.5) and np.allclose(r[-2:], 0.0)


def test_box_only_objects_keep_exact_vertices_and_zero_bounds():
    ms = configs.cad_set(10, 2, 3000.0, 1, 0)
    for o in range(ms.n):
        if cad.CATEGORIES[(o // 2) % len(cad.CATEGORIES)] not in ("shelf", "bed"):
            continue
        for lod in range(ms.n_lods - 1):
            assert (ms.hd_of(lod, o) == 0).all() and (ms.ph_of(lod, o) == 0).all()


@pytest.mark.parametrize("cat_index", [0, 3])     # table, lamp: cylinders
def test_cylinder_hausdorff_bounds_by_sampling(cat_index):
    ms = configs.cad_set(5, 1, 200.0, 2, 0)
    o = cat_index
    fine = ms.triangles(ms.n_lods - 1, o).astype(np.float64)
    rng = np.random.default_rng(cat_index)
    for lod in (0, 1):
        coarse = ms.triangles(lod, o).astype(np.float64)
        hd = ms.hd_of(lod, o).astype(np.float64)
        ph = ms.ph_of(lod, o).astype(np.float64)
        assert (hd > 0).any()
        # hd: points of coarse facets lie within hd of the fine surface
        for f in rng.choice(coarse.shape[0], 30, replace=False):
            tri = coarse[f]
            for a, b in ((1 / 3, 1 / 3), (0.5, 0.0), (0.0, 0.5), (0.45, 0.45)):
                p = tri[0] + a * (tri[1] - tri[0]) + b * (tri[2] - tri[0])
                assert oracle.point_mesh_dist(p, fine) <= hd[f] + 1e-9
        # ph: fine points lie within ph(f') of some coarse facet f'
        pick = rng.choice(fine.shape[0], 60, replace=False)
        w = rng.dirichlet((1.0, 1.0, 1.0), size=60)
        pts = np.vstack([fine.reshape(-1, 3)[::11], np.einsum("ij,ijk->ik", w, fine[pick])])
        for p in pts:
            assert min(oracle.point_tri_dist(p, coarse[f]) - ph[f] for f in range(coarse.shape[0])) <= 1e-9


def test_replicas_are_exact_translates_and_chunks_match():
    whole = configs.cad_set(6, 4, 800.0, 3, 1)
    for j in range(6):
        base = whole.object_verts(2, 4 * j).astype(np.float64)
        for i in range(1, 4):
            v = whole.object_verts(2, 4 * j + i).astype(np.float64)
            d = v - base
            if cad.CATEGORIES[j % len(cad.CATEGORIES)] in ("shelf", "bed"):
                assert np.allclose(d, d[0], rtol=0, atol=0)     # box-only models: exact
            else:
                assert np.allclose(d, d[0], rtol=0, atol=1e-3)
    part = configs.cad_set(6, 4, 800.0, 3, 1, start=7, count=9)
    for lod in range(whole.n_lods):
        for k in range(9):
            o = 7 + k
            assert np.array_equal(part.object_verts(lod, k), whole.object_verts(lod, o))
            assert np.array_equal(part.object_faces(lod, k), whole.object_faces(lod, o))
            if lod < whole.n_lods - 1:
                assert np.array_equal(part.hd_of(lod, k), whole.hd_of(lod, o))


def test_hand_placed_replicas_distance():
    # two replicas of a box-only model: a gap of 0.75 along x is their exact
    # distance, and shifted to touch they meet (distance exactly 0)
    rng = np.random.default_rng(5)
    parts = cad.model_parts(rng, "bed")
    w = max(p[2][0] for p in parts)
    for gap in (0.75, 0.0):
        ms = cad.make_cad([parts, parts], [np.zeros(3), np.array([w + gap, 0.0, 0.0])])
        A = ms.triangles(2, 0)
        B = ms.triangles(2, 1)
        assert oracle.obj_dist(A, B) == gap


def test_lod_bounds_bracket_distances_on_a_small_join():
    R = configs.cad_set(5, 4, 120.0, 4, 0)
    S = configs.cad_set(5, 4, 120.0, 4, 1)
    r, s, d = oracle.join_within(R, S, 1.0)
    assert len(r) > 0
    for lod in (0, 1):
        lb, ub = oracle.pair_bounds(R, S, r, s, lod)
        assert (lb <= d + 1e-12).all() and (d <= ub + 1e-12).all()


def test_planted_mistake_dropped_cylinder_bound_is_caught():
    # hd without the chord term r (1 - cos(pi / m)): some point of a coarse
    # cylinder facet lies farther from the fine surface than that
    ms = configs.cad_set(5, 1, 200.0, 2, 0)
    o = 3      # lamp: cylinders only
    fine = ms.triangles(ms.n_lods - 1, o).astype(np.float64)
    coarse = ms.triangles(0, o).astype(np.float64)
    hd = ms.hd_of(0, o).astype(np.float64)
    r = [p for p in cad.model_parts(np.random.default_rng([2, 0, 3, 37]), "lamp")]
    chord = min(p[5] * (1 - np.cos(np.pi / cad.CYL_SEGMENTS[0])) for p in r)
    broken = 0
    for f in range(0, coarse.shape[0], 7):
        p = coarse[f].mean(axis=0)
        broken += oracle.point_mesh_dist(p, fine) > hd[f] - chord + 1e-9
    assert broken > 0
