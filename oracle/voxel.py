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

Readings where the paper is silent (also listed in the design notes):

* the voxel count is round(2 % of the original facets), at least 1 and at
  most the coarsest LoD's facet count (there is nothing finer to cluster);
* the initial centres are "uniformly sampled" vertices: the coarsest LoD's
  vertices (those its facets use, in order of first use) at the evenly
  spaced positions floor((j + 1/2) V / k), so the oracle needs no random
  stream;
* assignment ties go to the lower centre index; a centre left without
  members keeps its position;
* the input carries no facet correspondence across LoDs, so a facet of any
  LoD belongs to the voxel whose final centre is nearest to its centroid:
  the same k centres partition every LoD (consistent across LoDs by
  construction);
* a voxel anchor is the vertex of the voxel's original facets closest to
  the centre of the voxel's box (ties: first in facet order).
"""
from __future__ import annotations

import numpy as np

VOXEL_FRACTION = 0.02


def voxel_count(f_original: int, f_coarsest: int) -> int:
    """Voxels of an object with ``f_original`` facets at full resolution and
    ``f_coarsest`` at its coarsest LoD."""
    k = int(np.floor(VOXEL_FRACTION * f_original + 0.5))
    return max(1, min(k, int(f_coarsest)))


def centroids(tri) -> np.ndarray:
    """Facet centroids of triangles ``tri`` [F, 9] or [F, 3, 3]."""
    t = np.asarray(tri, np.float64).reshape(-1, 3, 3)
    return t.mean(axis=1)


def assign(cent, centres) -> np.ndarray:
    """Index of the nearest centre of each centroid (lower index on ties)."""
    cent = np.asarray(cent, np.float64)
    centres = np.asarray(centres, np.float64)
    d2 = ((cent[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
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
            if m.any():
                centres[j] = cent[m].mean(axis=0)
    return centres


def initial_centres(coarse_tri, k: int) -> np.ndarray:
    """k vertices of the coarsest LoD, evenly spaced over its vertices in
    order of first use by its facets."""
    v = np.asarray(coarse_tri, np.float64).reshape(-1, 3)
    _, first = np.unique(v, axis=0, return_index=True)
    verts = v[np.sort(first)]
    V = verts.shape[0]
    idx = np.floor((np.arange(k) + 0.5) * V / k).astype(np.int64)
    return verts[np.minimum(idx, V - 1)]


def voxelize(tris_by_lod):
    """Voxels of one object from its triangles per LoD (``tris_by_lod[0]`` the
    coarsest, ``[-1]`` the original surfaces; each [F_l, 9]).

    Returns a dict: ``centres`` [k, 3]; ``labels`` (the voxel of every facet,
    one array per LoD); ``boxes`` [k, 6] (lo, hi of the voxel's original
    facets; +inf / -inf for a voxel without original facets); ``anchors``
    [k, 3] (nan for such a voxel)."""
    coarse = np.asarray(tris_by_lod[0], np.float64).reshape(-1, 9)
    orig = np.asarray(tris_by_lod[-1], np.float64).reshape(-1, 9)
    k = voxel_count(orig.shape[0], coarse.shape[0])
    centres = kmeans(centroids(coarse), initial_centres(coarse, k))
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
        anchors[j] = members[np.argmin(((members - c) ** 2).sum(axis=1))]
    return {"centres": centres, "labels": labels, "boxes": boxes, "anchors": anchors}


def box_mindist(a, b) -> float:
    """Minimum distance between the boxes a, b = (lo.xyz, hi.xyz): the
    length of the per-axis gaps (0 where the boxes overlap on an axis)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    g = np.maximum(0.0, np.maximum(b[:3] - a[3:], a[:3] - b[3:]))
    return float(np.sqrt((g * g).sum()))


def voxel_pair_bounds(vr, vs):
    """Algorithm 1 for one object pair: for voxel i of r and j of s,
    lb = MINDIST of their boxes, ub = distance of their anchors; voxels
    without original facets take no part (inf).  Returns (vpLB [nr, ns],
    vpUB [nr, ns], opLB, opUB)."""
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
            ub[i, j] = float(np.linalg.norm(vr["anchors"][i] - vs["anchors"][j]))
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
