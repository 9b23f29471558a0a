"""CPU FP64 oracle for the polyhedral spatial join -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library under ``paper_2604_19982_gb300``
never does: its join runs in CUDA kernels only.

The arithmetic lives in ``oracle.c`` (plain C, double precision, built with
``-ffp-contract=off``); this module only marshals :class:`synth.MeshSet`
inputs into flat triangle soups and calls it through ctypes.

Functions and the passages they follow (arXiv 2604.19982):

* :func:`tri_dist`      -- triangle-triangle distance (section 2.2); 0 exactly
                           when the closed triangles meet (:func:`tri_meet`,
                           exact orientation signs)
* :func:`obj_dist`      -- d(P1, P2) by brute force (section 2.1)
* :func:`pair_bounds`   -- Eq. 1 / Eq. 2 LoD bounds of object pairs
* :func:`join_within`   -- within-tau / intersection join (section 3)
* :func:`join_knn`      -- k-NN join, ties broken by object id (section 3)

``oracle.voxel`` holds the voxelization and voxel-pair filtering of
sections 2.1 and 3.2 (Algorithms 1 and 2) in numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (portable C, no ISA flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        i64p = C.POINTER(C.c_int64)
        i32p = C.POINTER(C.c_int32)
        L.or_tri_dist.restype = C.c_double
        L.or_tri_dist.argtypes = [dp, dp, dp]
        L.or_tri_dist_batch.restype = None
        L.or_tri_dist_batch.argtypes = [dp, dp, C.c_int64, dp, dp]
        L.or_point_tri_dist.restype = C.c_double
        L.or_point_tri_dist.argtypes = [dp, dp]
        L.or_point_mesh_dist.restype = C.c_double
        L.or_point_mesh_dist.argtypes = [dp, fp, C.c_int64]
        L.or_obj_dist.restype = C.c_double
        L.or_obj_dist.argtypes = [fp, C.c_int64, fp, C.c_int64]
        L.or_lod_bounds.restype = None
        L.or_lod_bounds.argtypes = [fp, fp, fp, C.c_int64, fp, fp, fp, C.c_int64, dp, dp]
        L.or_join.restype = C.c_int64
        L.or_join.argtypes = [C.c_int64, fp, i64p, C.c_int64, fp, i64p, C.c_int, C.c_double, C.c_int,
                              C.c_int, i64p, C.c_int64, C.c_int,
                              C.POINTER(i32p), C.POINTER(dp), C.POINTER(i64p)]
        L.or_free.restype = None
        L.or_free.argtypes = [C.c_void_p]
        L.or_tri_meet.restype = C.c_int
        L.or_tri_meet.argtypes = [dp, dp]
        for nm in ("or_orient3d_exact", "or_orient3d"):
            getattr(L, nm).restype = C.c_int
            getattr(L, nm).argtypes = [dp, dp, dp, dp]
        L.or_orient2d_exact.restype = C.c_int
        L.or_orient2d_exact.argtypes = [dp, dp, dp]
        L.or_pairs.restype = None
        L.or_pairs.argtypes = [fp, i64p, fp, fp, fp, i64p, fp, fp, i32p, i32p, C.c_int64, C.c_int, dp, dp]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


# ------------------------------------------------------------ marshalling


def soup(ms, lod: int | None = None):
    """De-indexed triangles of every object at ``lod`` (default: original):
    ``(tri float32 [nf_total, 9], off int64 [n+1], hd float32, ph float32)``."""
    lod = ms.n_lods - 1 if lod is None else lod
    V = ms.verts[lod]
    vo = ms.vert_off[lod]
    if ms.face_off[lod] is None:
        F = ms.faces[lod]
        nf = F.shape[0]
        idx = vo[:-1, None, None] + F[None, :, :]
        tri = V[idx].reshape(-1, 9)
        off = np.arange(ms.n + 1, dtype=np.int64) * nf
    else:
        fo = ms.face_off[lod]
        counts = np.diff(fo)
        base = np.repeat(vo[:-1], counts)
        tri = V[ms.faces[lod] + base[:, None]].reshape(-1, 9)
        off = fo.astype(np.int64)
    nf_tot = int(off[-1])
    hd = ms.hd[lod] if ms.hd[lod] is not None else np.zeros(nf_tot, np.float32)
    ph = ms.ph[lod] if ms.ph[lod] is not None else np.zeros(nf_tot, np.float32)
    return (np.ascontiguousarray(tri, np.float32), np.ascontiguousarray(off, np.int64),
            np.ascontiguousarray(hd, np.float32), np.ascontiguousarray(ph, np.float32))


# ------------------------------------------------------------ primitives


def tri_dist(P, Q):
    """Distances and closest points of triangle pairs: ``P, Q`` [n, 3, 3]."""
    P = np.ascontiguousarray(P, np.float64).reshape(-1, 9)
    Q = np.ascontiguousarray(Q, np.float64).reshape(-1, 9)
    n = P.shape[0]
    d = np.empty(n, np.float64)
    cp = np.empty((n, 6), np.float64)
    lib().or_tri_dist_batch(_p(P, C.c_double), _p(Q, C.c_double), n, _p(d, C.c_double), _p(cp, C.c_double))
    return d, cp.reshape(n, 2, 3)


def tri_meet(P, Q) -> bool:
    """Do the closed triangles ``P``, ``Q`` [3, 3] share a point?  Decided by
    exact orientation signs (the meeting test of :func:`tri_dist`)."""
    P = np.ascontiguousarray(P, np.float64).reshape(9)
    Q = np.ascontiguousarray(Q, np.float64).reshape(9)
    return bool(lib().or_tri_meet(_p(P, C.c_double), _p(Q, C.c_double)))


def orient3d(a, b, c, d, exact_only: bool = False) -> int:
    """Sign of (b - a) . ((c - a) x (d - a)) for double inputs: filtered
    (default) or by the integer path alone."""
    v = [np.ascontiguousarray(x, np.float64).reshape(3) for x in (a, b, c, d)]
    f = lib().or_orient3d_exact if exact_only else lib().or_orient3d
    return int(f(*[_p(x, C.c_double) for x in v]))


def orient2d_exact(a, b, c) -> int:
    """Sign of (b - a) x (c - a) for 2-D double inputs, integer path."""
    v = [np.ascontiguousarray(x, np.float64).reshape(2) for x in (a, b, c)]
    return int(lib().or_orient2d_exact(*[_p(x, C.c_double) for x in v]))


def point_tri_dist(p, T) -> float:
    p = np.ascontiguousarray(p, np.float64)
    T = np.ascontiguousarray(T, np.float64).reshape(9)
    return lib().or_point_tri_dist(_p(p, C.c_double), _p(T, C.c_double))


def point_mesh_dist(p, tri) -> float:
    p = np.ascontiguousarray(p, np.float64)
    tri = np.ascontiguousarray(tri, np.float32).reshape(-1, 9)
    return lib().or_point_mesh_dist(_p(p, C.c_double), _p(tri, C.c_float), tri.shape[0])


def obj_dist(A, B) -> float:
    """d(A, B) for two triangle soups [na, 3, 3] / [nb, 3, 3] (float32)."""
    A = np.ascontiguousarray(A, np.float32).reshape(-1, 9)
    B = np.ascontiguousarray(B, np.float32).reshape(-1, 9)
    return lib().or_obj_dist(_p(A, C.c_float), A.shape[0], _p(B, C.c_float), B.shape[0])


def lod_bounds(A, hdA, phA, B, hdB, phB):
    A = np.ascontiguousarray(A, np.float32).reshape(-1, 9)
    B = np.ascontiguousarray(B, np.float32).reshape(-1, 9)
    hdA, phA, hdB, phB = (np.ascontiguousarray(x, np.float32) for x in (hdA, phA, hdB, phB))
    lb, ub = C.c_double(), C.c_double()
    lib().or_lod_bounds(_p(A, C.c_float), _p(hdA, C.c_float), _p(phA, C.c_float), A.shape[0],
                        _p(B, C.c_float), _p(hdB, C.c_float), _p(phB, C.c_float), B.shape[0],
                        C.byref(lb), C.byref(ub))
    return lb.value, ub.value


# ------------------------------------------------------------ pair lists


def pair_dists(R, S, pr, ps, threads=None, soups=None):
    """Exact full-resolution d(r, s) of explicit pairs."""
    (tA, oA, _, _), (tB, oB, _, _) = soups or (soup(R), soup(S))
    pr = np.ascontiguousarray(pr, np.int32)
    ps = np.ascontiguousarray(ps, np.int32)
    n = pr.shape[0]
    lb = np.empty(n)
    ub = np.empty(n)
    lib().or_pairs(_p(tA, C.c_float), _p(oA, C.c_int64), None, None, _p(tB, C.c_float), _p(oB, C.c_int64),
                   None, None, _p(pr, C.c_int32), _p(ps, C.c_int32), n, threads or default_threads(),
                   _p(lb, C.c_double), _p(ub, C.c_double))
    return lb


def pair_bounds(R, S, pr, ps, lod: int, threads=None):
    """Eq. 2 lower / Eq. 1 upper bound of explicit pairs at one LoD."""
    tA, oA, hA, pA = soup(R, lod)
    tB, oB, hB, pB = soup(S, lod)
    pr = np.ascontiguousarray(pr, np.int32)
    ps = np.ascontiguousarray(ps, np.int32)
    n = pr.shape[0]
    lb = np.empty(n)
    ub = np.empty(n)
    lib().or_pairs(_p(tA, C.c_float), _p(oA, C.c_int64), _p(hA, C.c_float), _p(pA, C.c_float),
                   _p(tB, C.c_float), _p(oB, C.c_int64), _p(hB, C.c_float), _p(pB, C.c_float),
                   _p(pr, C.c_int32), _p(ps, C.c_int32), n, threads or default_threads(),
                   _p(lb, C.c_double), _p(ub, C.c_double))
    return lb, ub


# ------------------------------------------------------------ joins


def _join(R, S, pred, tau, k, prune, rlist, threads, soups=None):
    (tA, oA, _, _), (tB, oB, _, _) = soups or (soup(R), soup(S))
    rl = None if rlist is None else np.ascontiguousarray(rlist, np.int64)
    nr = R.n if rl is None else rl.shape[0]
    s_ptr = C.POINTER(C.c_int32)()
    d_ptr = C.POINTER(C.c_double)()
    c_ptr = C.POINTER(C.c_int64)()
    total = lib().or_join(R.n, _p(tA, C.c_float), _p(oA, C.c_int64), S.n, _p(tB, C.c_float), _p(oB, C.c_int64),
                          pred, float(tau), int(k), int(prune), _p(rl, C.c_int64), nr, threads or default_threads(),
                          C.byref(s_ptr), C.byref(d_ptr), C.byref(c_ptr))
    s = np.ctypeslib.as_array(s_ptr, shape=(max(total, 1),))[:total].copy()
    d = np.ctypeslib.as_array(d_ptr, shape=(max(total, 1),))[:total].copy()
    cnt = np.ctypeslib.as_array(c_ptr, shape=(max(nr, 1),))[:nr].copy()
    L = lib()
    L.or_free(C.cast(s_ptr, C.c_void_p))
    L.or_free(C.cast(d_ptr, C.c_void_p))
    L.or_free(C.cast(c_ptr, C.c_void_p))
    rid = np.arange(R.n, dtype=np.int64) if rl is None else rl
    r = np.repeat(rid, cnt).astype(np.int32)
    return r, s.astype(np.int32), d


def join_within(R, S, tau: float, prune: bool = True, rlist=None, threads=None, soups=None):
    """All (r, s) with d(r, s) <= tau, ordered by r (then ``rlist`` order) and s.

    Returns ``(r int32, s int32, d float64)``."""
    return _join(R, S, 0, tau, 0, prune, rlist, threads, soups)


def join_knn(R, S, k: int, rlist=None, threads=None, soups=None):
    """For each r the first min(k, |S|) objects of S under the key (d, id).

    Returns ``(r int32, s int32, d float64)`` grouped by r, each group sorted
    by (d, s)."""
    return _join(R, S, 1, 0.0, k, True, rlist, threads, soups)
