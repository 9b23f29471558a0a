"""Seeded synthetic polyhedra with levels of detail (LoDs) and facet-level
Hausdorff bounds.

This module only *makes inputs*: closed triangle meshes, their coarse LoDs and
the two per-facet error bounds the refinement stage consumes (``hd`` and
``ph``, section 2.1, "Facet-Level Hausdorff Bounds", Eq. 1-2).  It contains no
triangle-distance code, no bound application and no join decision, so it can
feed both the CUDA path and the CPU oracle without sharing any of the method's
arithmetic.

Shapes (stand-ins for the paper's pathology nuclei and vessels, section 4.1):

* blob: icosphere at subdivision ``sub`` (20*4**sub facets) whose radius is
  ``R * max(0.2, 1 + sum_lm c_lm Y_lm(u))`` with real orthonormal spherical
  harmonics of degree <= 4, ``R ~ lognormal(0, 0.25)``, ``c_lm ~ N(0, 0.05)``.
  Coarse LoDs are lower subdivisions of the same radial function, so their
  vertices are a prefix of the fine vertex array.
* tube: a circle of 16 segments (radius 2) swept along a Catmull-Rom spline
  through a 6-point random walk, rescaled to arc length ``L ~ U[50, 800]``,
  with ``n = 63 + 2 (L - 50)`` rings (32 n facets incl. the two centre-fan
  caps).  Coarse LoDs keep every 2nd / 4th ring plus the last.

Hausdorff bounds.  The paper defers the definitions of ``hd(f', P)`` and
``ph(P, f')`` to TDBase; what Eq. 1 and Eq. 2 need is (i) every point of a
coarse facet ``f'`` lies within ``hd(f')`` of the fine surface ``P`` and
(ii) every point of ``P`` lies within ``ph(f')`` of some coarse facet ``f'``
whose region covers it.  Both follow from a piecewise-affine correspondence
``phi`` between the coarse and fine surfaces over a common parameter domain:
on each fine parameter triangle ``T`` the fine surface is affine, and the
coarse facet's flat map ``A`` extends affinely, so ``|A - phi|`` is convex on
``T`` and peaks at ``T``'s vertices.  Hence
``max over fine vertices v whose triangles meet f' of |A(param(v)) - v|``
bounds both directed distances and we store it for both ``hd`` and ``ph``,
computed in float64 on the float32-rounded vertices and rounded *up* to
float32.  At full resolution ``hd = ph = 0``.
"""
from __future__ import annotations

import dataclasses
import math
from functools import lru_cache

import numpy as np

# --------------------------------------------------------------------------
# container


@dataclasses.dataclass
class MeshSet:
    """A set of closed triangle meshes with ``n_lods`` levels of detail.

    LoD 0 is the coarsest, LoD ``n_lods-1`` the original surface.  Per LoD:

    * ``verts[l]``  float32 [nv_total, 3]; ``vert_off[l]`` int64 [n+1].
    * ``faces[l]``  int32 [nf_total, 3] object-local vertex ids, or, when
      ``face_off[l] is None``, one shared template [nf, 3] used by every object.
    * ``hd[l]`` / ``ph[l]`` float32 [nf_total] (``None`` at the last LoD: 0).
    * ``anchor`` float32 [n, 3]: one vertex of the original surface per object.
    """

    n: int
    n_lods: int
    verts: list
    vert_off: list
    faces: list
    face_off: list
    hd: list
    ph: list
    anchor: np.ndarray
    kind: str = "mesh"

    # ---- derived helpers (host-side, used by tests and the oracle wrapper)
    def n_faces(self, lod: int, obj: int) -> int:
        if self.face_off[lod] is None:
            return int(self.faces[lod].shape[0])
        return int(self.face_off[lod][obj + 1] - self.face_off[lod][obj])

    def object_faces(self, lod: int, obj: int) -> np.ndarray:
        if self.face_off[lod] is None:
            return self.faces[lod]
        a, b = self.face_off[lod][obj], self.face_off[lod][obj + 1]
        return self.faces[lod][a:b]

    def object_verts(self, lod: int, obj: int) -> np.ndarray:
        a, b = self.vert_off[lod][obj], self.vert_off[lod][obj + 1]
        return self.verts[lod][a:b]

    def triangles(self, lod: int, obj: int) -> np.ndarray:
        """De-indexed triangles [nf, 3, 3] float32 of one object."""
        return self.object_verts(lod, obj)[self.object_faces(lod, obj)]

    def face_range(self, lod: int, obj: int):
        if self.face_off[lod] is None:
            nf = self.faces[lod].shape[0]
            return obj * nf, (obj + 1) * nf
        return int(self.face_off[lod][obj]), int(self.face_off[lod][obj + 1])

    def hd_of(self, lod: int, obj: int) -> np.ndarray:
        a, b = self.face_range(lod, obj)
        if self.hd[lod] is None:
            return np.zeros(b - a, np.float32)
        return self.hd[lod][a:b]

    def ph_of(self, lod: int, obj: int) -> np.ndarray:
        a, b = self.face_range(lod, obj)
        if self.ph[lod] is None:
            return np.zeros(b - a, np.float32)
        return self.ph[lod][a:b]

    def mbb(self) -> np.ndarray:
        """float32 [n, 6] (min xyz, max xyz) of the original surface."""
        L = self.n_lods - 1
        v = self.verts[L]
        off = self.vert_off[L]
        out = np.empty((self.n, 6), np.float32)
        if self.n == 0:
            return out
        # vertex counts may differ per object; reduceat handles ragged ranges
        starts = off[:-1]
        out[:, 0:3] = np.minimum.reduceat(v, starts, axis=0)
        out[:, 3:6] = np.maximum.reduceat(v, starts, axis=0)
        return out

    def total_faces(self, lod: int) -> int:
        if self.face_off[lod] is None:
            return self.n * int(self.faces[lod].shape[0])
        return int(self.face_off[lod][-1])


def concat(sets) -> MeshSet:
    """One MeshSet holding the objects of ``sets`` in order (same LoD count;
    a LoD with shared topology must use one template in every part)."""
    sets = list(sets)
    L = sets[0].n_lods
    verts, voff, faces, foff, hd, ph = [], [], [], [], [], []
    for l in range(L):
        shared = sets[0].face_off[l] is None
        # LoDs that share one vertex array in every part keep sharing it
        same_v = [next((m for m in range(l) if x.verts[m] is x.verts[l]), None) for x in sets]
        if same_v[0] is not None and all(v == same_v[0] for v in same_v):
            verts.append(verts[same_v[0]])
            voff.append(voff[same_v[0]])
        else:
            verts.append(np.concatenate([x.verts[l] for x in sets]))
            offs = [np.asarray(sets[0].vert_off[l], np.int64)]
            for x in sets[1:]:
                offs.append(np.asarray(x.vert_off[l][1:], np.int64) + offs[-1][-1])
            voff.append(np.concatenate(offs))
        if shared:
            faces.append(sets[0].faces[l])
            foff.append(None)
        else:
            faces.append(np.concatenate([x.faces[l] for x in sets]))
            offs = [np.asarray(sets[0].face_off[l], np.int64)]
            for x in sets[1:]:
                offs.append(np.asarray(x.face_off[l][1:], np.int64) + offs[-1][-1])
            foff.append(np.concatenate(offs))
        hd.append(None if sets[0].hd[l] is None else np.concatenate([x.hd[l] for x in sets]))
        ph.append(None if sets[0].ph[l] is None else np.concatenate([x.ph[l] for x in sets]))
    return MeshSet(n=sum(x.n for x in sets), n_lods=L, verts=verts, vert_off=voff, faces=faces, face_off=foff,
                   hd=hd, ph=ph, anchor=np.concatenate([x.anchor for x in sets]), kind=sets[0].kind)


def subset(ms: MeshSet, ids) -> MeshSet:
    """The objects ``ids`` of ``ms`` (in that order) as a MeshSet of their own."""
    ids = np.asarray(ids, np.int64)
    L = ms.n_lods
    verts, voff, faces, foff, hd, ph = [], [], [], [], [], []
    for l in range(L):
        same = next((m for m in range(l) if ms.verts[m] is ms.verts[l] and ms.vert_off[m] is ms.vert_off[l]), None)
        if same is not None:
            verts.append(verts[same])
            voff.append(voff[same])
        else:
            vo = np.asarray(ms.vert_off[l], np.int64)
            cnt = vo[ids + 1] - vo[ids]
            verts.append(np.concatenate([ms.verts[l][vo[i]:vo[i + 1]] for i in ids]) if len(ids)
                         else np.zeros((0, 3), np.float32))
            voff.append(np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64))
        if ms.face_off[l] is None:
            nf = ms.faces[l].shape[0]
            fo = np.arange(ms.n + 1, dtype=np.int64) * nf
            faces.append(ms.faces[l])
            foff.append(None)
        else:
            fo = np.asarray(ms.face_off[l], np.int64)
            cnt = fo[ids + 1] - fo[ids]
            faces.append(np.concatenate([ms.faces[l][fo[i]:fo[i + 1]] for i in ids]) if len(ids)
                         else np.zeros((0, 3), np.int32))
            foff.append(np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64))
        pick = (lambda a: None if a is None else
                (np.concatenate([a[fo[i]:fo[i + 1]] for i in ids]) if len(ids) else a[:0]))
        hd.append(pick(ms.hd[l]))
        ph.append(pick(ms.ph[l]))
    return MeshSet(n=len(ids), n_lods=L, verts=verts, vert_off=voff, faces=faces, face_off=foff, hd=hd, ph=ph,
                   anchor=np.ascontiguousarray(ms.anchor[ids]), kind=ms.kind)


# --------------------------------------------------------------------------
# icosphere with a hierarchical face order (children of face f are 4f..4f+3)


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], np.int64)
    return v, f


@lru_cache(maxsize=None)
def icosphere(sub: int):
    """Unit icosphere at subdivision ``sub``.

    Returns ``(dirs float64 [V,3], faces int32 [20*4**sub, 3])``.  Vertices of
    subdivision ``k`` are a prefix of those of ``k+1``; the four children of
    face ``f`` are faces ``4f .. 4f+3``.
    """
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    faces = f
    for _ in range(sub):
        mid = {}
        new_faces = np.empty((faces.shape[0] * 4, 3), np.int64)

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = (np.asarray(verts[a]) + np.asarray(verts[b])) / 2.0
                p = p / np.linalg.norm(p)
                mid[key] = len(verts)
                verts.append(tuple(p))
            return mid[key]

        for i, (a, b, c) in enumerate(faces):
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_faces[4 * i + 0] = (a, ab, ca)
            new_faces[4 * i + 1] = (ab, b, bc)
            new_faces[4 * i + 2] = (ca, bc, c)
            new_faces[4 * i + 3] = (ab, bc, ca)
        faces = new_faces
    return np.asarray(verts, np.float64), faces.astype(np.int32)


@lru_cache(maxsize=None)
def subdivision_map(sub_coarse: int, sub_fine: int):
    """Fine vertices inside each coarse face, with their barycentric position.

    Returns ``(ids int32 [Fc, K], bary float64 [Fc, K, 3])`` where ``K`` is the
    number of grid points of a triangle subdivided ``sub_fine - sub_coarse``
    times.  ``bary`` is w.r.t. the coarse face's three vertices, so the flat
    (coarse) position of fine vertex ``ids[f, k]`` is
    ``bary[f, k] @ coarse_face_verts``.  The descendants of coarse face ``f``
    are the fine faces ``f * 4**depth .. (f+1) * 4**depth - 1``.
    """
    _, fc = icosphere(sub_coarse)
    depth = sub_fine - sub_coarse
    tables = [icosphere(sub_coarse + d)[1] for d in range(depth + 1)]
    E = np.eye(3)
    ids_l, bary_l = [], []
    for f in range(fc.shape[0]):
        bary = {int(fc[f, k]): E[k] for k in range(3)}
        lo, hi = f, f + 1                      # descendant range at this level
        for d in range(depth):
            nxt = tables[d + 1]
            for i in range(lo, hi):
                a, b, c = (int(x) for x in tables[d][i])
                ab, ca = int(nxt[4 * i][1]), int(nxt[4 * i][2])
                bc = int(nxt[4 * i + 1][2])
                bary.setdefault(ab, (bary[a] + bary[b]) / 2.0)
                bary.setdefault(bc, (bary[b] + bary[c]) / 2.0)
                bary.setdefault(ca, (bary[c] + bary[a]) / 2.0)
            lo, hi = 4 * lo, 4 * hi
        keys = sorted(bary)
        ids_l.append(keys)
        bary_l.append([bary[k] for k in keys])
    return np.asarray(ids_l, np.int32), np.asarray(bary_l, np.float64)


# --------------------------------------------------------------------------
# real orthonormal spherical harmonics, degree <= 4 (25 functions)


def real_sh_deg4(u: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics Y_lm, l = 0..4, at unit vectors.

    ``u`` float64 [V, 3] -> [V, 25], ordered (l, m) with m = -l..l.
    """
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    pi = math.pi
    s = math.sqrt
    cols = [
        0.5 * s(1 / pi) * np.ones_like(x),
        s(3 / (4 * pi)) * y, s(3 / (4 * pi)) * z, s(3 / (4 * pi)) * x,
        0.5 * s(15 / pi) * x * y,
        0.5 * s(15 / pi) * y * z,
        0.25 * s(5 / pi) * (3 * z * z - 1),
        0.5 * s(15 / pi) * x * z,
        0.25 * s(15 / pi) * (x * x - y * y),
        0.25 * s(35 / (2 * pi)) * y * (3 * x * x - y * y),
        0.5 * s(105 / pi) * x * y * z,
        0.25 * s(21 / (2 * pi)) * y * (5 * z * z - 1),
        0.25 * s(7 / pi) * z * (5 * z * z - 3),
        0.25 * s(21 / (2 * pi)) * x * (5 * z * z - 1),
        0.25 * s(105 / pi) * z * (x * x - y * y),
        0.25 * s(35 / (2 * pi)) * x * (x * x - 3 * y * y),
        0.75 * s(35 / pi) * x * y * (x * x - y * y),
        0.75 * s(35 / (2 * pi)) * y * z * (3 * x * x - y * y),
        0.75 * s(5 / pi) * x * y * (7 * z * z - 1),
        0.75 * s(5 / (2 * pi)) * y * z * (7 * z * z - 3),
        (3 / 16) * s(1 / pi) * (35 * z ** 4 - 30 * z * z + 3),
        0.75 * s(5 / (2 * pi)) * x * z * (7 * z * z - 3),
        (3 / 8) * s(5 / pi) * (x * x - y * y) * (7 * z * z - 1),
        0.75 * s(35 / (2 * pi)) * x * z * (x * x - 3 * y * y),
        (3 / 16) * s(35 / pi) * (x * x * (x * x - 3 * y * y) - y * y * (3 * x * x - y * y)),
    ]
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# rounding helpers


def round_up_f32(x64: np.ndarray) -> np.ndarray:
    """float64 -> float32 rounded toward +inf, after a 1e-12 relative pad
    that absorbs the float64 rounding of the displacement computation."""
    x = np.asarray(x64, np.float64) * (1.0 + 1e-12)
    f = x.astype(np.float32)
    low = f.astype(np.float64) < x
    f[low] = np.nextafter(f[low], np.float32(np.inf))
    return f


# --------------------------------------------------------------------------
# blobs


def _blob_params(rng: np.random.Generator, count: int):
    R = rng.lognormal(0.0, 0.25, size=count)
    C = rng.normal(0.0, 0.05, size=(count, 25))
    return R, C


def make_blobs(centres: np.ndarray, R: np.ndarray, C: np.ndarray, subs):
    """Build a blob MeshSet from per-object centre, radius and SH coefficients.

    ``subs``: increasing icosphere subdivisions, one per LoD (last = original).
    Vertex storage is float32; faces use one shared template per LoD.
    """
    n = centres.shape[0]
    s_fine = subs[-1]
    dirs, _ = icosphere(s_fine)
    V = dirs.shape[0]
    Y = real_sh_deg4(dirs)                              # [V, 25]
    radial = R[:, None] * np.maximum(0.2, 1.0 + C @ Y.T)  # [n, V]
    X = centres[:, None, :] + radial[:, :, None] * dirs[None, :, :]
    Xf = X.astype(np.float32)                           # [n, V, 3]
    verts_all = Xf.reshape(n * V, 3)
    voff = np.arange(n + 1, dtype=np.int64) * V

    faces, hd, ph = [], [], []
    X64 = Xf.astype(np.float64)
    for li, s in enumerate(subs):
        _, f = icosphere(s)
        faces.append(f)
        if li == len(subs) - 1:
            hd.append(None)
            ph.append(None)
            continue
        ids, bary = subdivision_map(s, s_fine)          # [Fc, K], [Fc, K, 3]
        hdv = np.empty((n, f.shape[0]), np.float64)
        step = max(1, 4_000_000 // (f.shape[0] * ids.shape[1] * 3))
        for a in range(0, n, step):
            b = min(n, a + step)
            cv = X64[a:b][:, f]                           # [B, Fc, 3, 3]
            flat = np.einsum("fkc,bfcx->bfkx", bary, cv)  # [B, Fc, K, 3]
            act = X64[a:b][:, ids]                        # [B, Fc, K, 3]
            disp = np.sqrt(((act - flat) ** 2).sum(-1)).max(-1)
            hdv[a:b] = disp
        hv = round_up_f32(hdv).reshape(-1)
        hd.append(hv)
        ph.append(hv.copy())

    # anchor: the original-surface vertex closest to the MBB centre
    mn, mx = Xf.min(axis=1), Xf.max(axis=1)
    ctr = (mn.astype(np.float64) + mx) / 2.0
    d2 = ((X64 - ctr[:, None, :]) ** 2).sum(-1)
    anchor = Xf[np.arange(n), d2.argmin(axis=1)]

    L = len(subs)
    return MeshSet(n=n, n_lods=L, verts=[verts_all] * L, vert_off=[voff] * L,
                   faces=faces, face_off=[None] * L, hd=hd, ph=ph,
                   anchor=np.ascontiguousarray(anchor), kind="blob")


# --------------------------------------------------------------------------
# tubes


TUBE_SEGMENTS = 16
TUBE_RADIUS = 2.0


def tube_rings(L: float) -> int:
    """Number of sweep samples for arc length ``L`` (32 n facets in all)."""
    return int(63 + 2 * round(L - 50.0))


def _catmull_rom(P: np.ndarray, samples: int) -> np.ndarray:
    """Uniform Catmull-Rom through control points (end points duplicated)."""
    Q = np.vstack([P[:1], P, P[-1:]])
    segs = P.shape[0] - 1
    out = []
    for i in range(segs):
        p0, p1, p2, p3 = Q[i], Q[i + 1], Q[i + 2], Q[i + 3]
        t = np.linspace(0.0, 1.0, samples, endpoint=(i == segs - 1))[:, None]
        out.append(0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t * t
                          + (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3))
    return np.vstack(out)


def _tube_centerline(rng: np.random.Generator, centre: np.ndarray, L: float, n: int):
    # 6-point persistent random walk
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    pts = [np.zeros(3)]
    for _ in range(5):
        nd = d + 0.9 * rng.normal(size=3)
        d = nd / np.linalg.norm(nd)
        pts.append(pts[-1] + d)
    P = np.asarray(pts)
    dense = _catmull_rom(P, 512)
    seg = np.linalg.norm(np.diff(dense, axis=0), axis=1)
    arc = np.concatenate([[0.0], np.cumsum(seg)])
    scale = L / arc[-1]
    dense = dense * scale
    arc = arc * scale
    tgt = np.linspace(0.0, arc[-1], n)
    C = np.stack([np.interp(tgt, arc, dense[:, k]) for k in range(3)], axis=1)
    mn, mx = C.min(0), C.max(0)
    C = C - (mn + mx) / 2.0 + centre
    return C


def _tube_surface(C: np.ndarray):
    """Ring vertices [n, 16, 3] (float64) of the swept circle along ``C``."""
    n = C.shape[0]
    T = np.gradient(C, axis=0)
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    a = np.array([1.0, 0.0, 0.0]) if abs(T[0, 0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    N = np.empty_like(C)
    nv = a - (a @ T[0]) * T[0]
    N[0] = nv / np.linalg.norm(nv)
    for i in range(1, n):
        nv = N[i - 1] - (N[i - 1] @ T[i]) * T[i]
        N[i] = nv / math.sqrt(nv @ nv)
    B = np.cross(T, N)
    phi = 2.0 * np.pi * np.arange(TUBE_SEGMENTS) / TUBE_SEGMENTS
    ring = (np.cos(phi)[None, :, None] * N[:, None, :] + np.sin(phi)[None, :, None] * B[:, None, :])
    return C[:, None, :] + TUBE_RADIUS * ring


def _tube_lod_rings(n: int, step: int) -> np.ndarray:
    keep = list(range(0, n, step))
    if keep[-1] != n - 1:
        keep.append(n - 1)
    return np.asarray(keep, np.int64)


def _tube_faces(m: int) -> np.ndarray:
    """Faces of a tube with ``m`` rings: cap fan, side strips, cap fan.

    Vertex ``16 j + a`` is ring ``j`` angle ``a``; ``16 m`` / ``16 m + 1`` are
    the start / end cap centres.  Facets are ordered along the sweep.
    """
    S = TUBE_SEGMENTS
    a = np.arange(S)
    b = (a + 1) % S
    c0, c1 = S * m, S * m + 1
    cap0 = np.stack([np.full(S, c0), b, a], axis=1)
    j = np.arange(m - 1)[:, None]
    t1 = np.stack([S * j + a, S * (j + 1) + a, S * (j + 1) + b], axis=-1)   # [m-1, S, 3]
    t2 = np.stack([S * j + a, S * (j + 1) + b, S * j + b + 0 * j], axis=-1)
    sides = np.stack([t1, t2], axis=2).reshape(-1, 3)                       # per quad: T1, T2
    cap1 = np.stack([np.full(S, c1), S * (m - 1) + a, S * (m - 1) + b], axis=1)
    return np.vstack([cap0, sides, cap1]).astype(np.int32)


def _tube_hd(ringsF: np.ndarray, keep: np.ndarray) -> np.ndarray:
    """Displacement bound of the coarse tube facets w.r.t. the fine tube.

    Parameter domain: (u = fine ring index, v = angle index).  Each coarse
    quad between kept rings i0 < i1 at angle a is split into
    T1 = (i0,a),(i1,a),(i1,a+1) and T2 = (i0,a),(i1,a+1),(i0,a+1), like the
    fine quads.  The bound of a coarse triangle is the max, over the fine
    vertices of the strip [i0, i1] x {a, a+1} (the vertices of every fine
    triangle meeting it), of |A(u, v) - X(u, v)| with A the coarse triangle's
    affine map extended to the strip.
    """
    S = TUBE_SEGMENTS
    m = keep.shape[0]
    out = np.zeros(32 * m, np.float64)    # caps stay 0 (identical at all LoDs)
    side = np.zeros((m - 1, S, 2), np.float64)
    spans = np.diff(keep)
    A = np.arange(S)
    B = (A + 1) % S
    for span in np.unique(spans):
        qs = np.nonzero(spans == span)[0]
        i0 = keep[qs]                                     # [Q]
        i1 = i0 + span
        js = i0[:, None] + np.arange(span + 1)[None, :]   # [Q, J]
        uu = (np.arange(span + 1) / float(span))[None, :, None, None]
        X0 = ringsF[js][:, :, A]                          # [Q, J, S, 3]
        X1 = ringsF[js][:, :, B]
        P00 = ringsF[i0][:, None, A]                      # [Q, 1, S, 3]
        P10 = ringsF[i1][:, None, A]
        P11 = ringsF[i1][:, None, B]
        P01 = ringsF[i0][:, None, B]
        A1v0 = P00 + uu * (P10 - P00)
        A1v1 = A1v0 + (P11 - P10)
        h1 = np.maximum(np.linalg.norm(A1v0 - X0, axis=-1).max(1), np.linalg.norm(A1v1 - X1, axis=-1).max(1))
        A2v0 = P00 + uu * (P11 - P01)
        A2v1 = A2v0 + (P01 - P00)
        h2 = np.maximum(np.linalg.norm(A2v0 - X0, axis=-1).max(1), np.linalg.norm(A2v1 - X1, axis=-1).max(1))
        side[qs, :, 0] = h1
        side[qs, :, 1] = h2
    out[S:S + 2 * S * (m - 1)] = side.reshape(-1)
    return out


def make_tubes(rng_for, centres: np.ndarray, lengths: np.ndarray, steps=(4, 2, 1)):
    """Build a tube MeshSet; ``rng_for(i)`` returns the generator of tube i."""
    n = centres.shape[0]
    L_ = len(steps)
    verts = [[] for _ in range(L_)]
    faces = [[] for _ in range(L_)]
    hd = [[] for _ in range(L_)]
    vcount = [[0] for _ in range(L_)]
    fcount = [[0] for _ in range(L_)]
    anchors = np.empty((n, 3), np.float32)
    for i in range(n):
        rng = rng_for(i)
        nr = tube_rings(float(lengths[i]))
        C = _tube_centerline(rng, centres[i], float(lengths[i]), nr)
        rings = _tube_surface(C)
        ringsF = rings.astype(np.float32)
        capsF = np.stack([C[0], C[-1]]).astype(np.float32)
        rings64 = ringsF.astype(np.float64)
        fine_all = np.vstack([ringsF.reshape(-1, 3), capsF])
        mn, mx = fine_all.min(0).astype(np.float64), fine_all.max(0).astype(np.float64)
        ctr = (mn + mx) / 2.0
        anchors[i] = fine_all[((fine_all.astype(np.float64) - ctr) ** 2).sum(1).argmin()]
        for li, st in enumerate(steps):
            keep = _tube_lod_rings(nr, st)
            m = keep.shape[0]
            v = np.vstack([ringsF[keep].reshape(-1, 3), capsF])
            verts[li].append(v)
            faces[li].append(_tube_faces(m))
            vcount[li].append(vcount[li][-1] + v.shape[0])
            fcount[li].append(fcount[li][-1] + 32 * m)
            if li < L_ - 1:
                hd[li].append(_tube_hd(rings64, keep))
    out_v, out_f, out_vo, out_fo, out_hd, out_ph = [], [], [], [], [], []
    for li in range(L_):
        out_v.append(np.ascontiguousarray(np.vstack(verts[li]) if n else np.zeros((0, 3), np.float32)))
        out_f.append(np.ascontiguousarray(np.vstack(faces[li]) if n else np.zeros((0, 3), np.int32)))
        out_vo.append(np.asarray(vcount[li], np.int64))
        out_fo.append(np.asarray(fcount[li], np.int64))
        if li < L_ - 1:
            hv = round_up_f32(np.concatenate(hd[li]) if n else np.zeros(0))
            out_hd.append(hv)
            out_ph.append(hv.copy())
        else:
            out_hd.append(None)
            out_ph.append(None)
    return MeshSet(n=n, n_lods=L_, verts=out_v, vert_off=out_vo, faces=out_f,
                   face_off=out_fo, hd=out_hd, ph=out_ph, anchor=anchors, kind="tube")


# --------------------------------------------------------------------------
# generic helpers used by tests (hand-made meshes)


def from_triangles(tris_per_object, n_lods: int = 1) -> MeshSet:
    """MeshSet from explicit per-object triangle lists [nf, 3, 3] (one LoD,
    replicated ``n_lods`` times with zero Hausdorff bounds)."""
    verts, faces, vo, fo = [], [], [0], [0]
    for t in tris_per_object:
        t = np.asarray(t, np.float32).reshape(-1, 3, 3)
        verts.append(t.reshape(-1, 3))
        faces.append(np.arange(t.shape[0] * 3, dtype=np.int32).reshape(-1, 3))
        vo.append(vo[-1] + t.shape[0] * 3)
        fo.append(fo[-1] + t.shape[0])
    V = np.ascontiguousarray(np.vstack(verts)) if verts else np.zeros((0, 3), np.float32)
    F = np.ascontiguousarray(np.vstack(faces)) if faces else np.zeros((0, 3), np.int32)
    vo, fo = np.asarray(vo, np.int64), np.asarray(fo, np.int64)
    anchor = np.asarray([np.asarray(t, np.float32).reshape(-1, 3)[0] for t in tris_per_object],
                        np.float32).reshape(-1, 3)
    z = [np.zeros(int(fo[-1]), np.float32) for _ in range(n_lods - 1)] + [None]
    return MeshSet(n=len(tris_per_object), n_lods=n_lods, verts=[V] * n_lods, vert_off=[vo] * n_lods,
                   faces=[F] * n_lods, face_off=[fo] * n_lods, hd=z, ph=[None if x is None else x.copy() for x in z],
                   anchor=anchor, kind="explicit")


def box_triangles(lo, hi) -> np.ndarray:
    """The 12 triangles of an axis-aligned box surface."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    c = np.array([[lo[0] if i & 1 == 0 else hi[0], lo[1] if i & 2 == 0 else hi[1],
                   lo[2] if i & 4 == 0 else hi[2]] for i in range(8)])
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    tris = []
    for a, b, cc, d in quads:
        tris.append([c[a], c[b], c[cc]])
        tris.append([c[a], c[cc], c[d]])
    return np.asarray(tris, np.float64)
