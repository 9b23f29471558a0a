"""CAD-like synthetic objects: the stand-in for the paper's second workload,
ModelNet40's pre-aligned CAD models replicated 100 times and shifted to
different locations (section 4.1, datasets T and I, joined as TI / TT).
No model of that suite is reproduced: every model here is a furniture-like
assembly drawn from a seeded generator of our own -- axis-aligned boxes
(slabs, panels, frames) and upright cylinders (legs, poles, shades).

Levels of detail (three, coarsest first):

* boxes: every face an n x n grid of quads, n = 1, 2, 4, each quad split
  along the same diagonal.  Box coordinates lie on a 1/64 grid and the grid
  lines on a 1/256 grid, exact in float32, so the coarse and fine surfaces
  are the same point set facet for facet: hd = ph = 0;
* cylinders: m = 8, 16, 32 segments on the same axial rings (the coarse
  angles are a subset of the fine ones), centre-fan caps.  The coarse
  polygon lies inside the fine one and both inside the circle, so moving a
  point radially (in the cap plane for caps) between the two surfaces
  travels at most r (1 - cos(pi / m)): that bounds hd and ph of every facet
  of a coarse cylinder, plus twice the float32 rounding of the vertices
  (sqrt(3) |x|max 2^-24 each), rounded up to float32.

A model is replicated ``replicas`` times; replica i of model j is the model
shifted by a translation on the 1/64 grid (uniform in the cube), so
replicas are exact translates.  Objects are ordered model-major.
"""
from __future__ import annotations

import math

import numpy as np

from .mesh import MeshSet, round_up_f32

BOX_GRID = (1, 2, 4)
CYL_SEGMENTS = (8, 16, 32)
GRID = 1.0 / 64.0
RING_SPACING = 4.0       # axial ring spacing of cylinders (at most)
CATEGORIES = ("table", "chair", "shelf", "lamp", "bed")


def _q(x):
    """Round to the 1/64 grid."""
    return np.round(np.asarray(x, np.float64) / GRID) * GRID


# ----------------------------------------------------------------- parts

def box_mesh(lo, hi, n: int):
    """Closed surface of the box [lo, hi]: vertices [V, 3] (float64, exact
    dyadics) and faces [F, 3]; each face an n x n grid, quads split along
    the diagonal from their (u0, v0) to their (u1, v1) corner."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    tris = []
    t = np.arange(n + 1) / n
    for axis in range(3):
        u_ax, v_ax = [a for a in range(3) if a != axis]
        for side in (lo[axis], hi[axis]):
            P = np.empty((n + 1, n + 1, 3))
            P[..., axis] = side
            P[..., u_ax] = (lo[u_ax] + t * (hi[u_ax] - lo[u_ax]))[:, None]
            P[..., v_ax] = (lo[v_ax] + t * (hi[v_ax] - lo[v_ax]))[None, :]
            for i in range(n):
                for j in range(n):
                    a, b, c, d = P[i, j], P[i + 1, j], P[i + 1, j + 1], P[i, j + 1]
                    tris.append((a, b, c))
                    tris.append((a, c, d))
    T = np.asarray(tris)
    V, inv = np.unique(T.reshape(-1, 3), axis=0, return_inverse=True)
    return V, inv.reshape(-1, 3).astype(np.int32)


def cylinder_mesh(cx, cy, z0, z1, r, m: int):
    """Closed upright cylinder: m segments at the angles 2 pi k / m, axial
    rings every RING_SPACING at most, centre-fan caps.  Returns vertices
    (float64) and faces."""
    h = max(1, int(math.ceil((z1 - z0) / RING_SPACING)))
    zs = z0 + (z1 - z0) * np.arange(h + 1) / h
    ang = 2.0 * np.pi * np.arange(m) / m
    ring = np.stack([cx + r * np.cos(ang), cy + r * np.sin(ang)], axis=1)
    V = [np.column_stack([ring, np.full(m, z)]) for z in zs]
    V.append(np.array([[cx, cy, z0], [cx, cy, z1]]))
    V = np.vstack(V)
    c0, c1 = (h + 1) * m, (h + 1) * m + 1
    F = []
    for a in range(h):
        for k in range(m):
            k1 = (k + 1) % m
            p, q, s, t = a * m + k, a * m + k1, (a + 1) * m + k1, (a + 1) * m + k
            F.append((p, q, s))
            F.append((p, s, t))
    for k in range(m):
        k1 = (k + 1) % m
        F.append((c0, k1, k))
        F.append((c1, h * m + k, h * m + k1))
    return V, np.asarray(F, np.int32)


# ----------------------------------------------------------------- models

def model_parts(rng: np.random.Generator, category: str):
    """Parts of one model at the origin: ("box", lo, hi) and ("cyl", cx, cy,
    z0, z1, r), coordinates on the 1/64 grid."""
    u = lambda a, b: float(_q(rng.uniform(a, b)))
    parts = []
    if category in ("table", "chair"):
        w, d = u(12, 40), u(10, 30)
        hgt = u(10, 30) if category == "table" else u(8, 18)
        top = u(1, 3)
        parts.append(("box", (0.0, 0.0, hgt), (w, d, hgt + top)))
        r = u(0.5, 1.5)
        for x in (r + 0.5, w - r - 0.5):
            for y in (r + 0.5, d - r - 0.5):
                parts.append(("cyl", float(_q(x)), float(_q(y)), 0.0, hgt, r))
        if category == "chair":
            back = u(10, 25)
            parts.append(("box", (0.0, d - top, hgt + top), (w, d, hgt + top + back)))
    elif category == "shelf":
        w, d, hgt = u(20, 50), u(8, 20), u(30, 60)
        t = u(1, 2.5)
        parts.append(("box", (0.0, 0.0, 0.0), (t, d, hgt)))
        parts.append(("box", (w - t, 0.0, 0.0), (w, d, hgt)))
        k = int(rng.integers(2, 6))
        for i in range(k):
            z = float(_q(i * (hgt - t) / (k - 1)))
            parts.append(("box", (t, 0.0, z), (w - t, d, z + t)))
    elif category == "lamp":
        rb, hb = u(4, 8), u(1, 2)
        parts.append(("cyl", 0.0, 0.0, 0.0, hb, rb))
        hp = u(20, 50)
        parts.append(("cyl", 0.0, 0.0, hb, hb + hp, u(0.5, 1.0)))
        parts.append(("cyl", 0.0, 0.0, hb + hp, hb + hp + u(6, 12), u(5, 10)))
    elif category == "bed":
        w, d = u(30, 50), u(60, 90)
        parts.append(("box", (0.0, 0.0, 0.0), (w, d, u(6, 12))))
        top = float(parts[0][2][2])
        parts.append(("box", (1.0, 1.0, top), (w - 1.0, d - 1.0, top + u(4, 8))))
        parts.append(("box", (0.0, d - 2.0, 0.0), (w, d, top + u(15, 30))))
    else:
        raise ValueError(category)
    return parts


def _lod_mesh(parts, shift, li: int):
    """Vertices (float32), faces and per-facet hd (float64) of one object at
    LoD li, its parts shifted by `shift`."""
    Vs, Fs, H = [], [], []
    nv = 0
    for p in parts:
        if p[0] == "box":
            V, F = box_mesh(np.asarray(p[1]) + shift, np.asarray(p[2]) + shift, BOX_GRID[li])
            h = np.zeros(F.shape[0])
        else:
            _, cx, cy, z0, z1, r = p
            m = CYL_SEGMENTS[li]
            V, F = cylinder_mesh(cx + shift[0], cy + shift[1], z0 + shift[2], z1 + shift[2], r, m)
            geo = 0.0 if li == len(CYL_SEGMENTS) - 1 else r * (1.0 - math.cos(math.pi / m))
            h = np.full(F.shape[0], geo)
        Vs.append(V)
        Fs.append(F + nv)
        H.append(h)
        nv += V.shape[0]
    V = np.vstack(Vs)
    Vf = V.astype(np.float32)
    F = np.vstack(Fs).astype(np.int32)
    H = np.concatenate(H)
    return Vf, F, H


def make_cad(models, shifts, n_lods: int = 3) -> MeshSet:
    """MeshSet of objects (parts list, shift) = zip(models, shifts)."""
    L = n_lods
    assert L == len(BOX_GRID)
    verts = [[] for _ in range(L)]
    faces = [[] for _ in range(L)]
    hds = [[] for _ in range(L)]
    vcount = [[0] for _ in range(L)]
    fcount = [[0] for _ in range(L)]
    n = len(models)
    anchors = np.empty((n, 3), np.float32)
    for o, (parts, shift) in enumerate(zip(models, shifts)):
        shift = np.asarray(shift, np.float64)
        # box vertices on the 1/256 grid stay exact in float32 below 2^15
        assert np.all(np.abs(shift) < 2.0 ** 14), "CAD objects must lie within |x| < 16384"
        per = [_lod_mesh(parts, shift, li) for li in range(L)]
        fineV = per[-1][0].astype(np.float64)
        mx = max(float(np.abs(x[0]).max()) for x in per)
        # float32 rounding of a vertex moves it by at most sqrt(3) |x|max 2^-24
        slack = 2.0 * math.sqrt(3.0) * mx * 2.0 ** -24
        lo, hi = fineV.min(0), fineV.max(0)
        anchors[o] = per[-1][0][((fineV - (lo + hi) / 2.0) ** 2).sum(1).argmin()]
        for li, (Vf, F, H) in enumerate(per):
            verts[li].append(Vf)
            faces[li].append(F)
            vcount[li].append(vcount[li][-1] + Vf.shape[0])
            fcount[li].append(fcount[li][-1] + F.shape[0])
            if li < L - 1:
                hds[li].append(np.where(H > 0, H + slack, 0.0))
    out_hd, out_ph = [], []
    for li in range(L):
        if li < L - 1:
            hv = round_up_f32(np.concatenate(hds[li]) if n else np.zeros(0))
            out_hd.append(hv)
            out_ph.append(hv.copy())
        else:
            out_hd.append(None)
            out_ph.append(None)
    return MeshSet(n=n, n_lods=L,
                   verts=[np.ascontiguousarray(np.vstack(v)) if n else np.zeros((0, 3), np.float32) for v in verts],
                   vert_off=[np.asarray(c, np.int64) for c in vcount],
                   faces=[np.ascontiguousarray(np.vstack(f)) if n else np.zeros((0, 3), np.int32) for f in faces],
                   face_off=[np.asarray(c, np.int64) for c in fcount],
                   hd=out_hd, ph=out_ph, anchor=anchors, kind="cad")
