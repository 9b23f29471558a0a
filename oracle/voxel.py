"""Voxels and voxel-pair filtering -- TEST INFRASTRUCTURE (oracle).

Only ``tests/`` may import this module; the library never does.  Plain
numpy in double precision, written from the paper (arXiv 2604.19982):

* :func:`voxel_count`  -- 2 % of an object's facets (section 4, configurations)
* :func:`kmeans`       -- k-means over facet centroids, two centroid updates
                          (section 2.1, "Object Voxelization")
* :func:`voxelize`     -- voxels of one object: clustered on its coarsest LoD
                          and shared by every LoD (section 2.1, "Consistent
                          Voxelization across LoDs"); voxel boxes and anchors
                          on the original surfaces (section 2.1, "Object and
                          Voxel Centers")
* :func:`box_mindist`  -- MINDIST of two axis-aligned boxes (the voxel-pair
                          lower bound of section 3.2)
* :func:`voxel_pair_bounds` -- Algorithm 1: every voxel pair's [lb, ub], and
                          their minima, the object pair's [lb, ub]
* :func:`decide_within`     -- object-pair pruning of section 3.2
* :func:`prune_voxel_pairs` -- Algorithm 2: the voxel pairs with lb <= the
                          object pair's ub, in the order of the count / scan
                          / compact kernels
* :func:`voxelize_set`, :func:`voxel_filter` -- the same over whole sets and
                          lists of object pairs (section 3.2's pipeline:
                          bounds, object-level decision, pruning)

Readings where the paper is silent (also listed in the design notes):

* the voxel count is round(2 % of the original facets), at least 1 and at
  most the coarsest LoD's facet count (there is nothing finer to cluster);
* the initial centres are "uniformly sampled" vertices: the polyhedron's
  vertices at its coarsest LoD, in the order its vertex array lists them,
  taken at the evenly spaced positions floor((j + 1/2) V / k), so the
  oracle needs no random stream;
* assignment ties go to the lower centre index; a centre left without
  members keeps its position;
* the input carries no facet correspondence across LoDs, so a facet of any
  LoD belongs to the voxel whose final centre is nearest to its centroid:
  the same k centres partition every LoD (consistent across LoDs by
  construction);
* a voxel anchor is the vertex of the voxel's original facets closest to
  the centre of the voxel's box (ties: first in facet order, then corner
  order).

Every floating-point expression is written out in a fixed order (sums of
three squares as (x^2 + y^2) + z^2, centroids as (v0 + v1) + v2 then / 3,
a centre as the running sum of its members in facet order, then / count),
with no fused multiply-add and no library reduction, so a kernel that
evaluates the same expressions in the same order reaches the same doubles.
"""
from __future__ import annotations

import math

import numpy as np

VOXEL_FRACTION = 0.02


def voxel_count(f_original: int, f_coarsest: int) -> int:
    """Voxels of an object with ``f_original`` facets at full resolution and
    ``f_coarsest`` at its coarsest LoD (none without coarsest facets: there
    is nothing to cluster)."""
    if f_coarsest <= 0:
        return 0
    k = int(np.floor(VOXEL_FRACTION * f_original + 0.5))
    return max(1, min(k, int(f_coarsest)))


def centroids(tri) -> np.ndarray:
    """Facet centroids of triangles ``tri`` [F, 9] or [F, 3, 3]:
    ((v0 + v1) + v2) / 3."""
    t = np.asarray(tri, np.float64).reshape(-1, 3, 3)
    return (t[:, 0] + t[:, 1] + t[:, 2]) / 3.0


def sq3(d) -> np.ndarray:
    """(x^2 + y^2) + z^2 over the last axis (length 3)."""
    return d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]


def assign(cent, centres) -> np.ndarray:
    """Index of the nearest centre of each centroid by squared distance
    (lower index on ties)."""
    cent = np.asarray(cent, np.float64)
    centres = np.asarray(centres, np.float64)
    d2 = sq3(cent[:, None, :] - centres[None, :, :])
    return np.argmin(d2, axis=1)   # argmin returns the first of equal minima


def kmeans(cent, init, updates: int = 2):
    """Lloyd's iterations: ``updates`` times, assign every centroid to its
    nearest centre, then move each centre to the mean of its members (a
    centre without members stays).  Returns the centres after the last
    update."""
    centres = np.array(init, np.float64, copy=True)
    cent = np.asarray(cent, np.float64)
    for _ in range(updates):
        lab = assign(cent, centres)
        for j in range(centres.shape[0]):
            m = lab == j
            cnt = int(m.sum())
            if cnt:
                # running sum in facet order (cumsum accumulates in order)
                centres[j] = np.cumsum(cent[m], axis=0)[-1] / float(cnt)
    return centres


def initial_centres(coarse_verts, k: int) -> np.ndarray:
    """k vertices of the polyhedron's vertex array at its coarsest LoD, at
    the evenly spaced positions floor((j + 1/2) V / k)."""
    verts = np.asarray(coarse_verts, np.float64).reshape(-1, 3)
    V = verts.shape[0]
    idx = np.floor((np.arange(k) + 0.5) * V / k).astype(np.int64)
    return verts[np.minimum(idx, V - 1)]


def voxelize(tris_by_lod, coarse_verts):
    """Voxels of one object from its triangles per LoD (``tris_by_lod[0]`` the
    coarsest, ``[-1]`` the original surfaces; each [F_l, 9]) and its vertex
    array at the coarsest LoD (``coarse_verts`` [V, 3]).

    Returns a dict: ``centres`` [k, 3]; ``labels`` (the voxel of every facet,
    one array per LoD); ``boxes`` [k, 6] (lo, hi of the voxel's original
    facets; +inf / -inf for a voxel without original facets); ``anchors``
    [k, 3] (nan for such a voxel)."""
    coarse = np.asarray(tris_by_lod[0], np.float64).reshape(-1, 9)
    orig = np.asarray(tris_by_lod[-1], np.float64).reshape(-1, 9)
    k = voxel_count(orig.shape[0], coarse.shape[0])
    if k == 0:
        return {"centres": np.zeros((0, 3)),
                "labels": [np.full(np.asarray(t).reshape(-1, 9).shape[0], -1, np.int64) for t in tris_by_lod],
                "boxes": np.zeros((0, 6)), "anchors": np.zeros((0, 3))}
    centres = kmeans(centroids(coarse), initial_centres(coarse_verts, k))
    labels = [assign(centroids(t), centres) for t in tris_by_lod]
    lab = labels[-1]
    boxes = np.empty((k, 6))
    boxes[:, :3] = np.inf
    boxes[:, 3:] = -np.inf
    anchors = np.full((k, 3), np.nan)
    pts = orig.reshape(-1, 3, 3)
    for j in range(k):
        members = pts[lab == j].reshape(-1, 3)
        if members.shape[0] == 0:
            continue
        boxes[j, :3] = members.min(axis=0)
        boxes[j, 3:] = members.max(axis=0)
        c = 0.5 * (boxes[j, :3] + boxes[j, 3:])
        anchors[j] = members[np.argmin(sq3(members - c))]
    return {"centres": centres, "labels": labels, "boxes": boxes, "anchors": anchors}


def box_mindist(a, b) -> float:
    """Minimum distance between the boxes a, b = (lo.xyz, hi.xyz): the
    length of the per-axis gaps (0 where the boxes overlap on an axis)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    g = np.maximum(0.0, np.maximum(b[:3] - a[3:], a[:3] - b[3:]))
    return math.sqrt(float(sq3(g)))


def voxel_pair_bounds(vr, vs):
    """Algorithm 1 for one object pair: for voxel i of r and j of s,
    lb = MINDIST of their boxes, ub = distance of their anchors; voxels
    without original facets take no part (inf), and a pair with no voxel
    pair at all has opLB = opUB = inf.  Returns (vpLB [nr, ns], vpUB
    [nr, ns], opLB, opUB)."""
    nr, ns = vr["boxes"].shape[0], vs["boxes"].shape[0]
    lb = np.full((nr, ns), np.inf)
    ub = np.full((nr, ns), np.inf)
    for i in range(nr):
        if not np.isfinite(vr["boxes"][i, 0]):
            continue
        for j in range(ns):
            if not np.isfinite(vs["boxes"][j, 0]):
                continue
            lb[i, j] = box_mindist(vr["boxes"][i], vs["boxes"][j])
            ub[i, j] = math.sqrt(float(sq3(vr["anchors"][i] - vs["anchors"][j])))
    if lb.size == 0:      # an object without voxels: no voxel pair bounds it
        return lb, ub, math.inf, math.inf
    return lb, ub, float(lb.min()), float(ub.min())


def decide_within(op_lb: float, op_ub: float, tau: float) -> int:
    """Object-pair pruning for a within-tau query: 1 a result (ub <= tau),
    2 pruned (lb > tau), 0 undecided."""
    if op_ub <= tau:
        return 1
    if op_lb > tau:
        return 2
    return 0


def prune_voxel_pairs(vp_lb, op_ub: float) -> np.ndarray:
    """Algorithm 2 for one object pair: the voxel pairs (i, j) with
    lb <= the object pair's ub, in the order t = i * n_s + j that the count,
    scan and compact kernels keep.  Returns an int array [m, 2]."""
    lb = np.asarray(vp_lb, np.float64)
    ns = lb.shape[1]
    t = np.nonzero(lb.reshape(-1) <= op_ub)[0]
    return np.stack([t // ns, t % ns], axis=1).astype(np.int64)


def voxelize_set(ms):
    """:func:`voxelize` of every object of a mesh set (anything with ``n``,
    ``n_lods``, ``object_verts(lod, o)`` and ``object_faces(lod, o)``): a
    list, one dict per object."""
    out = []
    for o in range(ms.n):
        per_lod = []
        for lod in range(ms.n_lods):
            v = np.asarray(ms.object_verts(lod, o), np.float64)
            f = np.asarray(ms.object_faces(lod, o), np.int64)
            per_lod.append(v[f].reshape(-1, 9))
        out.append(voxelize(per_lod, np.asarray(ms.object_verts(0, o), np.float64)))
    return out


def voxel_filter(vox_r, vox_s, pr, ps, tau: float):
    """The voxel-pair filtering of section 3.2 for object pairs
    (pr[p], ps[p]) of two voxelized sets: Algorithm 1's bounds for every
    pair, the object-level decision (tau < 0: none, every pair stays
    undecided), and Algorithm 2's surviving voxel pairs of the undecided
    pairs.  Returns a dict of op_lb, op_ub [n]; status [n] (0 undecided,
    1 result, 2 pruned); vp_off [n + 1] and vp_lb, vp_ub (each pair's
    n_r x n_s block, row-major); kept_off [n + 1] and kept [m, 2]."""
    n = len(pr)
    op_lb = np.zeros(n)
    op_ub = np.zeros(n)
    status = np.zeros(n, np.uint8)
    vp_off = np.zeros(n + 1, np.int64)
    kept_off = np.zeros(n + 1, np.int64)
    vlb, vub, kept = [], [], []
    for p in range(n):
        vr, vs = vox_r[int(pr[p])], vox_s[int(ps[p])]
        lb, ub, olb, oub = voxel_pair_bounds(vr, vs)
        op_lb[p], op_ub[p] = olb, oub
        status[p] = decide_within(olb, oub, tau) if tau >= 0 else 0
        vlb.append(lb.reshape(-1))
        vub.append(ub.reshape(-1))
        vp_off[p + 1] = vp_off[p] + lb.size
        kp = prune_voxel_pairs(lb, oub) if status[p] == 0 else np.zeros((0, 2), np.int64)
        kept.append(kp)
        kept_off[p + 1] = kept_off[p] + kp.shape[0]
    cat = (lambda xs, shape: np.concatenate(xs) if xs else np.zeros(shape))
    return {"op_lb": op_lb, "op_ub": op_ub, "status": status, "vp_off": vp_off,
            "vp_lb": cat(vlb, (0,)), "vp_ub": cat(vub, (0,)), "kept_off": kept_off,
            "kept": cat(kept, (0, 2)).astype(np.int64).reshape(-1, 2)}
