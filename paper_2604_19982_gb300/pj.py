"""Thin ctypes binding of ``libpj.so`` (C ABI in ``include/pj.h``).

Argument marshalling only: every step of a join runs in the library's CUDA
kernels.  Importing this module loads the in-tree library and raises if it
is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import collections
import ctypes as C
import json
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpj.so")

PJ_OK, PJ_EINVAL, PJ_ENOMEM, PJ_ECUDA, PJ_ETIMEOUT, PJ_ENONFINITE, PJ_EBOUNDS, PJ_ECANCELLED, PJ_ESOURCE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
WITHIN, INTERSECT, KNN = 0, 1, 2
FP64, FP32 = 0, 1
EXACT_DIST, USE_MLP, USE_GRAPH, AUTOTUNE, TILE_PRUNE = 1, 2, 4, 8, 16
TUNED = USE_MLP | USE_GRAPH | AUTOTUNE | TILE_PRUNE
MAX_LODS = 8

_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_u8p = C.POINTER(C.c_uint8)


class MeshSetDesc(C.Structure):
    _fields_ = [("n_objects", C.c_int32), ("n_lods", C.c_int32),
                ("verts", _fp * MAX_LODS), ("vert_off", _i64p * MAX_LODS),
                ("faces", _i32p * MAX_LODS), ("face_off", _i64p * MAX_LODS),
                ("n_faces_shared", C.c_int32 * MAX_LODS),
                ("hd", _fp * MAX_LODS), ("ph", _fp * MAX_LODS), ("anchor", _fp)]


class Query(C.Structure):
    _fields_ = [("pred", C.c_int), ("tau", C.c_double), ("k", C.c_int32), ("prec", C.c_int),
                ("flags", C.c_uint32), ("timeout_s", C.c_double)]


class ResultC(C.Structure):
    _fields_ = [("n", C.c_int64), ("r", _i32p), ("s", _i32p), ("d_lo", _dp), ("d_hi", _dp), ("d", _dp),
                ("exact", _u8p), ("priv", C.c_void_p)]


FILL_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.POINTER(MeshSetDesc))

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        st = C.c_int
        sig = {
            "pj_create": (st, [C.POINTER(vp), C.c_int, C.c_char_p]),
            "pj_destroy": (None, [vp]),
            "pj_load_set": (st, [vp, C.POINTER(MeshSetDesc), C.POINTER(vp)]),
            "pj_load_set_streamed": (st, [vp, C.c_int64, C.c_int, FILL_FN, vp, C.POINTER(vp)]),
            "pj_free_set": (None, [vp]),
            "pj_join": (st, [vp, vp, vp, C.POINTER(Query), C.POINTER(ResultC)]),
            "pj_join_async": (st, [vp, vp, vp, C.POINTER(Query), vp, C.POINTER(ResultC)]),
            "pj_result_free": (None, [C.POINTER(ResultC)]),
            "pj_get_stats": (st, [vp, C.c_char_p, C.c_size_t]),
            "pj_mlp_train": (st, [vp, _fp, _fp, C.c_int64, C.c_int, C.c_uint64]),
            "pj_mlp_fit": (st, [vp, vp, vp, C.POINTER(Query), C.c_int64, C.c_int, C.c_uint64, _dp]),
            "pj_mlp_save": (st, [vp, C.c_char_p]),
            "pj_mlp_load": (st, [vp, C.c_char_p]),
            "pj_mlp_set_weights": (st, [vp, _fp, _fp, _fp, _fp, _fp, _fp]),
            "pj_mlp_get_weights": (st, [vp, _fp, _fp, _fp, _fp, _fp, _fp]),
            "pj_mlp_forward": (st, [vp, vp, C.c_int64, vp, vp]),
            "pj_mlp_grad": (st, [vp, vp, vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp]),
            "pj_pair_features": (st, [vp, vp, vp, _i32p, _i32p, C.c_int64, vp]),
            "pj_tri_dist": (st, [vp, vp, vp, C.c_int64, C.c_int, vp, vp, vp]),
            "pj_pair_bounds": (st, [vp, vp, vp, _i32p, _i32p, C.c_int64, C.c_int, C.c_int, _dp, _dp]),
            "pj_fma_peak": (st, [vp, C.c_int, _dp]),
            "pj_pair_bounds_static": (st, [vp, vp, vp, vp, vp, C.c_int64, C.c_int, C.c_int, vp, vp, vp]),
            "pj_voxel_count": (st, [vp, _i64p]),
            "pj_voxels_read": (st, [vp, vp, _i64p, _dp, _fp, _fp]),
            "pj_voxel_labels_read": (st, [vp, vp, C.c_int, _i32p]),
            "pj_voxel_filter": (st, [vp, vp, vp, vp, vp, C.c_int64, C.c_double, C.c_int, vp, vp, vp, vp, vp, vp,
                                     C.c_int64, vp, vp, _i64p, vp]),
            "pj_chunk_file_write": (st, [C.c_char_p, C.POINTER(MeshSetDesc)]),
            "pj_chunk_source_open": (st, [C.POINTER(C.c_char_p), C.c_int, C.c_int, C.POINTER(vp)]),
            "pj_chunk_source_info": (st, [vp, _i64p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "pj_chunk_source_fill": (st, [vp, C.c_int, C.POINTER(MeshSetDesc)]),
            "pj_chunk_source_stats": (st, [vp, C.c_char_p, C.c_size_t]),
            "pj_chunk_source_close": (None, [vp]),
            "pj_last_error": (C.c_char_p, [vp]),
            "pj_status_str": (C.c_char_p, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class Cancel(Exception):
    """Raised by a streamed set's chunk function to cancel the join."""


class PJError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{lib().pj_status_str(status).decode()} ({status}): {msg}")
        self.status = status


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def _is_device(a) -> bool:
    return getattr(a, "is_cuda", False)


def describe(ms, keep: list) -> MeshSetDesc:
    """Fill a ``pj_mesh_set_desc`` from a mesh-set object with the attributes
    ``n, n_lods, verts, vert_off, faces, face_off, hd, ph, anchor``: numpy
    arrays, or (for a streamed set's chunks) contiguous CUDA tensors of the
    same dtype for verts, faces, hd, ph and anchor, which the library then
    reads in place.  Arrays made contiguous here are appended to ``keep``
    (they must outlive the call)."""
    d = MeshSetDesc()
    d.n_objects = int(ms.n)
    d.n_lods = int(ms.n_lods)

    def c(a, dt, ct):
        if _is_device(a):
            if not a.is_contiguous() or a.element_size() != np.dtype(dt).itemsize:
                raise ValueError("device arrays must be contiguous and of the host array's dtype")
            keep.append(a)
            return C.cast(C.c_void_p(a.data_ptr()), C.POINTER(ct)), int(a.shape[0])
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return _ptr(a, ct), int(a.shape[0])

    for lvl in range(ms.n_lods):
        d.verts[lvl] = c(ms.verts[lvl], np.float32, C.c_float)[0]
        d.vert_off[lvl] = c(ms.vert_off[lvl], np.int64, C.c_int64)[0]
        d.faces[lvl], nf = c(ms.faces[lvl], np.int32, C.c_int32)
        if ms.face_off[lvl] is None:
            d.face_off[lvl] = None
            d.n_faces_shared[lvl] = nf
        else:
            d.face_off[lvl] = c(ms.face_off[lvl], np.int64, C.c_int64)[0]
            d.n_faces_shared[lvl] = 0
        d.hd[lvl] = c(ms.hd[lvl], np.float32, C.c_float)[0] if ms.hd[lvl] is not None else None
        d.ph[lvl] = c(ms.ph[lvl], np.float32, C.c_float)[0] if ms.ph[lvl] is not None else None
    d.anchor = c(ms.anchor, np.float32, C.c_float)[0]
    return d


class Result:
    """Host copy of a ``pj_result`` (numpy arrays)."""

    def __init__(self, rc: ResultC):
        n = int(rc.n)
        self.n = n

        def arr(p, dt):
            if n == 0:
                return np.zeros(0, dt)
            return np.ctypeslib.as_array(p, shape=(n,)).astype(dt, copy=True)

        self.r = arr(rc.r, np.int32)
        self.s = arr(rc.s, np.int32)
        self.d_lo = arr(rc.d_lo, np.float64)
        self.d_hi = arr(rc.d_hi, np.float64)
        self.d = arr(rc.d, np.float64)
        self.exact = arr(rc.exact, np.uint8)

    def pairs(self):
        return list(zip(self.r.tolist(), self.s.tolist()))


def write_chunk_file(path: str, ms) -> None:
    """pj_chunk_file_write: one chunk (a mesh-set object of host arrays) to
    a chunk file."""
    keep = []
    d = describe(ms, keep)
    st = lib().pj_chunk_file_write(os.fsencode(path), C.byref(d))
    if st != PJ_OK:
        raise PJError(st, f"cannot write chunk file {path}")


class ChunkView:
    """Host copies of one chunk as a chunk source hands it out (the fields
    of a mesh-set object)."""

    def __init__(self, d: MeshSetDesc):
        n, L = int(d.n_objects), int(d.n_lods)
        self.n, self.n_lods = n, L
        arr = (lambda p, count, dt: np.ctypeslib.as_array(p, shape=(count,)).astype(dt, copy=True)
               if count > 0 else np.zeros(0, dt))
        self.verts, self.vert_off, self.faces, self.face_off, self.hd, self.ph = [], [], [], [], [], []
        for l in range(L):
            vo = arr(d.vert_off[l], n + 1, np.int64)
            self.vert_off.append(vo)
            self.verts.append(arr(d.verts[l], 3 * int(vo[-1]), np.float32).reshape(-1, 3))
            if d.face_off[l]:
                fo = arr(d.face_off[l], n + 1, np.int64)
                rows, nf = int(fo[-1]), int(fo[-1])
                self.face_off.append(fo)
            else:
                rows = int(d.n_faces_shared[l]) if n > 0 else 0
                nf = n * rows
                self.face_off.append(None)
            self.faces.append(arr(d.faces[l], 3 * rows, np.int32).reshape(-1, 3))
            self.hd.append(arr(d.hd[l], nf, np.float32) if d.hd[l] else None)
            self.ph.append(arr(d.ph[l], nf, np.float32) if d.ph[l] else None)
        self.anchor = arr(d.anchor, 3 * n, np.float32).reshape(-1, 3)


class ChunkSource:
    """pj_chunk_source_*: chunk files read ahead by a native thread; pass it
    to :meth:`Context.load_set_files`."""

    def __init__(self, paths, readahead: int = 2):
        self.paths = [os.fsencode(p) for p in paths]
        arr = (C.c_char_p * len(self.paths))(*self.paths)
        h = C.c_void_p()
        st = lib().pj_chunk_source_open(arr, len(self.paths), int(readahead), C.byref(h))
        if st != PJ_OK:
            raise PJError(st, "cannot open the chunk files")
        self.h = h.value
        n, c, L = C.c_int64(), C.c_int(), C.c_int()
        lib().pj_chunk_source_info(self.h, C.byref(n), C.byref(c), C.byref(L))
        self.n_objects, self.n_chunks, self.n_lods = n.value, c.value, L.value

    def chunk(self, c: int) -> ChunkView:
        """Ask for chunk c as a join would, and copy it out."""
        d = MeshSetDesc()
        st = lib().pj_chunk_source_fill(self.h, int(c), C.byref(d))
        if st != PJ_OK:
            raise PJError(st, f"chunk {c}")
        return ChunkView(d)

    def stats(self) -> dict:
        buf = C.create_string_buffer(1024)
        lib().pj_chunk_source_stats(self.h, buf, len(buf))
        return json.loads(buf.value.decode())

    def close(self):
        if self.h:
            lib().pj_chunk_source_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Set:
    def __init__(self, ctx: "Context", handle: int, n: int, n_lods: int):
        self.ctx = ctx
        self.handle = handle
        self.n = n
        self.n_lods = n_lods
        ctx._sets.add(self)

    def free(self):
        if self.handle:
            lib().pj_free_set(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    def __init__(self, device: int = 0, options: dict | None = None):
        h = C.c_void_p()
        opt = json.dumps(options).encode() if options else None
        st = lib().pj_create(C.byref(h), int(device), opt)
        if st != PJ_OK:
            raise PJError(st, "pj_create failed (no usable sm_103 GPU?)")
        self.h = h.value
        self._keep = []
        self._sets = weakref.WeakSet()

    def _check(self, st: int):
        if st != PJ_OK:
            raise PJError(st, (lib().pj_last_error(self.h) or b"").decode())

    def close(self):
        """Free the sets loaded through this context, then the context."""
        if self.h:
            for s in list(self._sets):
                s.free()
            lib().pj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sets
    def load_set(self, ms) -> Set:
        keep = []
        d = describe(ms, keep)
        h = C.c_void_p()
        self._check(lib().pj_load_set(self.h, C.byref(d), C.byref(h)))
        return Set(self, h.value, int(ms.n), int(ms.n_lods))

    def load_set_streamed(self, n_objects: int, n_chunks: int, chunk_fn) -> Set:
        """``chunk_fn(c)`` returns the mesh-set object of chunk ``c`` (called
        from the library's loader thread during a join); raising
        :class:`Cancel` stops the join with PJ_ECANCELLED, any other
        exception with PJ_ESOURCE."""
        # the arrays of the last two chunks stay referenced: the library may
        # still lay out chunk c while it fills chunk c + 1 (on its other
        # loader thread), and is done with it when it asks for chunk c + 2
        keep_box = collections.deque(maxlen=2)

        def fill(user, chunk, out):
            try:
                ms = chunk_fn(int(chunk))
                keep = []
                d = describe(ms, keep)
                keep_box.append((keep, d, ms))
                C.memmove(out, C.byref(d), C.sizeof(MeshSetDesc))
                return PJ_OK
            except Cancel:
                return PJ_ECANCELLED
            except Exception:   # any failure of the source
                return PJ_ESOURCE

        cb = FILL_FN(fill)
        h = C.c_void_p()
        self._check(lib().pj_load_set_streamed(self.h, int(n_objects), int(n_chunks), cb, None, C.byref(h)))
        s = Set(self, h.value, int(n_objects), 0)
        s._cb = cb
        s._keep = keep_box
        return s

    def load_set_files(self, src: ChunkSource) -> Set:
        """A set streamed from chunk files: pj_load_set_streamed with the
        source's native fill callback (the source must stay open while the
        set is joined)."""
        fill = C.cast(lib().pj_chunk_source_fill, FILL_FN)
        h = C.c_void_p()
        self._check(lib().pj_load_set_streamed(self.h, int(src.n_objects), int(src.n_chunks), fill,
                                               C.c_void_p(src.h), C.byref(h)))
        s = Set(self, h.value, int(src.n_objects), src.n_lods)
        s._cb = fill
        s._src = src
        return s

    # ---- joins
    def join(self, R: Set, S: Set, pred: int = WITHIN, tau: float = 0.0, k: int = 0, prec: int = FP64,
             flags: int = 0, timeout_s: float = 0.0, stream: int | None = None) -> Result:
        q = Query(pred, float(tau), int(k), int(prec), int(flags), float(timeout_s))
        rc = ResultC()
        if stream is None:
            st = lib().pj_join(self.h, R.handle, S.handle, C.byref(q), C.byref(rc))
        else:
            st = lib().pj_join_async(self.h, R.handle, S.handle, C.byref(q), C.c_void_p(stream), C.byref(rc))
        self._check(st)
        try:
            return Result(rc)
        finally:
            lib().pj_result_free(C.byref(rc))

    def stats(self) -> dict:
        buf = C.create_string_buffer(1 << 16)
        self._check(lib().pj_get_stats(self.h, buf, len(buf)))
        return json.loads(buf.value.decode())

    # ---- kernel-level entry points
    def tri_dist(self, P_dev: int, Q_dev: int, n: int, prec: int, out_dev: int, err_dev: int | None = None,
                 stream: int | None = None):
        self._check(lib().pj_tri_dist(self.h, C.c_void_p(P_dev), C.c_void_p(Q_dev), int(n), int(prec),
                                      C.c_void_p(out_dev), C.c_void_p(err_dev) if err_dev else None,
                                      C.c_void_p(stream) if stream else None))

    def pair_bounds(self, R: Set, S: Set, pr, ps, lod: int, prec: int):
        pr = np.ascontiguousarray(pr, np.int32)
        ps = np.ascontiguousarray(ps, np.int32)
        n = pr.shape[0]
        lb = np.empty(n)
        ub = np.empty(n)
        self._check(lib().pj_pair_bounds(self.h, R.handle, S.handle, _ptr(pr, C.c_int32), _ptr(ps, C.c_int32), n,
                                         int(lod), int(prec), _ptr(lb, C.c_double), _ptr(ub, C.c_double)))
        return lb, ub

    def pair_bounds_static(self, R: Set, S: Set, pr_dev: int, ps_dev: int, n: int, lod: int, prec: int,
                           lb_dev: int, ub_dev: int, stream: int | None = None):
        """pj_pair_bounds_static: device buffers in and out, no allocation."""
        self._check(lib().pj_pair_bounds_static(self.h, R.handle, S.handle, C.c_void_p(pr_dev), C.c_void_p(ps_dev),
                                                int(n), int(lod), int(prec), C.c_void_p(lb_dev), C.c_void_p(ub_dev),
                                                C.c_void_p(stream) if stream else None))

    # ---- voxels (context option "voxels": 1)
    def voxel_count(self, S: Set) -> int:
        v = C.c_int64()
        self._check(lib().pj_voxel_count(S.handle, C.byref(v)))
        return v.value

    def voxels(self, S: Set) -> dict:
        """A set's voxels: voxel_off [n + 1], centres [V, 3] (double), boxes
        [V, 6] and anchors [V, 3] (float32)."""
        V = self.voxel_count(S)
        off = np.empty(S.n + 1, np.int64)
        cen = np.empty((V, 3), np.float64)
        box = np.empty((V, 6), np.float32)
        anc = np.empty((V, 3), np.float32)
        self._check(lib().pj_voxels_read(self.h, S.handle, _ptr(off, C.c_int64), _ptr(cen, C.c_double),
                                         _ptr(box, C.c_float), _ptr(anc, C.c_float)))
        return {"voxel_off": off, "centres": cen, "boxes": box, "anchors": anc}

    def voxel_offsets(self, S: Set) -> np.ndarray:
        """voxel_off [n + 1] of a set's voxels."""
        off = np.empty(S.n + 1, np.int64)
        self._check(lib().pj_voxels_read(self.h, S.handle, _ptr(off, C.c_int64), None, None, None))
        return off

    def voxel_labels(self, S: Set, lod: int, n_facets: int) -> np.ndarray:
        """The object-local voxel of each of the n_facets facets of LoD lod."""
        lab = np.empty(int(n_facets), np.int32)
        self._check(lib().pj_voxel_labels_read(self.h, S.handle, int(lod), _ptr(lab, C.c_int32)))
        return lab

    def voxel_filter(self, R: Set, S: Set, pr_dev: int, ps_dev: int, n: int, tau: float, out: dict,
                     vp_cap: int, prec: int = FP64, stream: int | None = None) -> int:
        """pj_voxel_filter: device buffers in and out (``out`` maps op_lb,
        op_ub, status, vp_off, vp_lb, vp_ub, kept_off, kept to device
        addresses); returns the number of surviving voxel pairs."""
        nk = C.c_int64()
        d = [C.c_void_p(out[k]) for k in ("op_lb", "op_ub", "status", "vp_off", "vp_lb", "vp_ub")]
        self._check(lib().pj_voxel_filter(self.h, R.handle, S.handle, C.c_void_p(pr_dev), C.c_void_p(ps_dev), int(n),
                                          float(tau), int(prec), *d, int(vp_cap), C.c_void_p(out["kept_off"]),
                                          C.c_void_p(out["kept"]), C.byref(nk),
                                          C.c_void_p(stream) if stream else None))
        return nk.value

    def fma_peak(self, fp64: bool) -> float:
        """Measured FMA throughput in GFLOP/s (FMA = 2 flops)."""
        g = C.c_double()
        self._check(lib().pj_fma_peak(self.h, 1 if fp64 else 0, C.byref(g)))
        return g.value

    # ---- learned proposal
    def mlp_fit(self, R: Set, S: Set, pred: int = KNN, tau: float = 0.0, k: int = 0, max_pairs: int = 200000,
                epochs: int = 30, seed: int = 1) -> float:
        """pj_mlp_fit: train fresh proposal weights on a sample of the
        query's candidates; returns the held-out RMSE in log(1 + d)."""
        q = Query(pred, float(tau), int(k), FP32, 0, 0.0)
        rmse = C.c_double()
        self._check(lib().pj_mlp_fit(self.h, R.handle, S.handle, C.byref(q), int(max_pairs), int(epochs), int(seed),
                                     C.byref(rmse)))
        return rmse.value

    def mlp_train(self, feats, target, epochs: int = 20, seed: int = 0):
        feats = np.ascontiguousarray(feats, np.float32)
        target = np.ascontiguousarray(target, np.float32)
        self._check(lib().pj_mlp_train(self.h, _ptr(feats, C.c_float), _ptr(target, C.c_float), feats.shape[0],
                                       int(epochs), int(seed)))

    def mlp_set_weights(self, w1, b1, w2, b2, w3, b3):
        a = [np.ascontiguousarray(x, np.float32) for x in (w1, b1, w2, b2, w3, b3)]
        self._check(lib().pj_mlp_set_weights(self.h, *[_ptr(x, C.c_float) for x in a]))

    def mlp_get_weights(self):
        shapes = [(64, 16), (64,), (64, 64), (64,), (64,), (1,)]
        a = [np.empty(s, np.float32) for s in shapes]
        self._check(lib().pj_mlp_get_weights(self.h, *[_ptr(x, C.c_float) for x in a]))
        return a

    def mlp_save(self, path: str):
        self._check(lib().pj_mlp_save(self.h, path.encode()))

    def mlp_load(self, path: str):
        self._check(lib().pj_mlp_load(self.h, path.encode()))

    def mlp_forward(self, feats_dev: int, n: int, out_dev: int, stream: int | None = None):
        self._check(lib().pj_mlp_forward(self.h, C.c_void_p(feats_dev), int(n), C.c_void_p(out_dev),
                                         C.c_void_p(stream) if stream else None))

    def mlp_grad(self, feats_dev, target_dev, n, loss_dev, grads_dev, stream=None):
        g = [C.c_void_p(x) if x else None for x in grads_dev]
        self._check(lib().pj_mlp_grad(self.h, C.c_void_p(feats_dev), C.c_void_p(target_dev), int(n),
                                      C.c_void_p(loss_dev), *g, C.c_void_p(stream) if stream else None))

    def pair_features(self, R: Set, S: Set, pr, ps, out_dev: int):
        pr = np.ascontiguousarray(pr, np.int32)
        ps = np.ascontiguousarray(ps, np.int32)
        self._check(lib().pj_pair_features(self.h, R.handle, S.handle, _ptr(pr, C.c_int32), _ptr(ps, C.c_int32),
                                           pr.shape[0], C.c_void_p(out_dev)))
