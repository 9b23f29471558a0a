"""The five seeded synthetic workloads (stand-ins for the paper's digital
pathology nuclei/vessel sets, section 4.1 and Table "Dataset Parameters").

Every object is drawn from its own counter-keyed stream
(``numpy.random.default_rng([seed, set_id, block, ...])``) so any chunk of a
set can be regenerated independently of the others.

==========  ==========================  ==========================  =========
workload    R                           S                           predicate
==========  ==========================  ==========================  =========
blobs100    100 blobs, LoD sub 1,2      100 blobs, side 20          within 0.5
blobs20k    20,000 blobs, sub 1,2,3     20,000 blobs, side 400      tau 0 and 1
knn50k      50,000 blobs, GMM(20, 15)   50,000 blobs, side 1000     3-NN
tubes2k     2,000 tubes (3 LoDs)        200,000 blobs, side 2320    within 2
stream2m    2,000,000 blobs (64 chunks) 20,000 tubes, side 5000     within 1
cadTI       400 CAD-like models x 100   100 models x 100, side 1500 tau 0, 1
==========  ==========================  ==========================  =========

cadTI stands in for the paper's ModelNet T x I join (section 4.1): the
models are our own furniture-like assemblies (``synth.cad``), replicated
and shifted as the paper replicates its CAD models.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import cad
from .mesh import MeshSet, _blob_params, concat, make_blobs, make_tubes

BLOCK = 1024  # objects per random-stream block

BLOB_SUBS = (1, 2, 3)


def _rng(*key):
    return np.random.default_rng([int(k) & 0xFFFFFFFF for k in key])


def gmm_centres(seed: int, n_clusters: int, side: float) -> np.ndarray:
    """Mixture centres shared by R and S of one workload."""
    return _rng(seed, 991, n_clusters).uniform(0.0, side, size=(n_clusters, 3))


def blob_params(seed: int, set_id: int, start: int, count: int, side: float,
                gmm=None, sigma: float = 15.0):
    """Centres, radii and SH coefficients of blobs ``start .. start+count``."""
    cs, Rs, Cs = [], [], []
    first_block = start // BLOCK
    last_block = (start + count - 1) // BLOCK if count > 0 else first_block - 1
    for blk in range(first_block, last_block + 1):
        rng = _rng(seed, set_id, blk, 17)
        if gmm is None:
            c = rng.uniform(0.0, side, size=(BLOCK, 3))
        else:
            lab = rng.integers(0, gmm.shape[0], size=BLOCK)
            c = np.clip(gmm[lab] + rng.normal(0.0, sigma, size=(BLOCK, 3)), 0.0, side)
        R, C = _blob_params(rng, BLOCK)
        lo = max(start, blk * BLOCK) - blk * BLOCK
        hi = min(start + count, (blk + 1) * BLOCK) - blk * BLOCK
        cs.append(c[lo:hi])
        Rs.append(R[lo:hi])
        Cs.append(C[lo:hi])
    if not cs:
        return np.zeros((0, 3)), np.zeros(0), np.zeros((0, 25))
    return np.vstack(cs), np.concatenate(Rs), np.vstack(Cs)


def blob_set(n: int, side: float, seed: int, set_id: int, subs=BLOB_SUBS,
             start: int = 0, count: int | None = None, gmm=None, sigma: float = 15.0) -> MeshSet:
    count = n - start if count is None else count
    c, R, C = blob_params(seed, set_id, start, count, side, gmm, sigma)
    return make_blobs(c, R, C, subs)


def tube_params(n: int, side: float, seed: int, set_id: int, start: int = 0,
                count: int | None = None, length_range=(50.0, 800.0)):
    """Centres and arc lengths of tubes ``start .. start+count`` (cheap: no
    surface is built).  A tube's centre line has the centre as the middle of
    its box and at most its arc length as extent per axis, so the tube lies
    in the box centre +- (length / 2 + radius)."""
    count = n - start if count is None else count
    centres = np.empty((count, 3))
    lengths = np.empty(count)
    for i in range(count):
        rng = _rng(seed, set_id, start + i, 29)
        centres[i] = rng.uniform(0.0, side, size=3)
        lengths[i] = rng.uniform(*length_range)
    return centres, lengths


def tube_set(n: int, side: float, seed: int, set_id: int, start: int = 0,
             count: int | None = None, length_range=(50.0, 800.0)) -> MeshSet:
    """Tubes with centres uniform in the cube and arc lengths uniform in
    ``length_range`` (the workload's range by default; tests use shorter
    tubes to keep the oracle fast)."""
    centres, lengths = tube_params(n, side, seed, set_id, start, count, length_range)
    return make_tubes(lambda i: _rng(seed, set_id, start + i, 31), centres, lengths)


def tube_list(n: int, side: float, seed: int, set_id: int, ids, length_range=(50.0, 800.0)) -> MeshSet:
    """The tubes ``ids`` of a tube set, generated alone (each from its own
    stream), in that order."""
    parts = [tube_set(n, side, seed, set_id, start=int(i), count=1, length_range=length_range) for i in ids]
    return concat(parts) if parts else tube_set(n, side, seed, set_id, start=0, count=0)


def cad_set(n_models: int, replicas: int, side: float, seed: int, set_id: int, start: int = 0,
            count: int | None = None) -> MeshSet:
    """CAD-like objects (``synth.cad``): n_models furniture-like models
    (categories in turn), each replicated ``replicas`` times at translations
    on the 1/64 grid uniform in [0, side)^3; object o is replica
    o % replicas of model o // replicas (objects start .. start + count)."""
    n = n_models * replicas
    count = n - start if count is None else count
    models, shifts = [], []
    cache = {}
    for o in range(start, start + count):
        j, i = divmod(o, replicas)
        if j not in cache:
            cache[j] = cad.model_parts(_rng(seed, set_id, j, 37), cad.CATEGORIES[j % len(cad.CATEGORIES)])
        models.append(cache[j])
        shifts.append(cad._q(_rng(seed, set_id, j, i, 41).uniform(0.0, side, size=3)))
    return cad.make_cad(models, shifts)


@dataclasses.dataclass
class Workload:
    name: str
    R: MeshSet
    S: MeshSet
    pred: str            # "within" | "knn"
    taus: tuple = ()
    k: int = 0


def scaled_side(side: float, n_full: int, n: int) -> float:
    """Cube side that keeps the object density of the full-size workload."""
    return side * (n / n_full) ** (1.0 / 3.0)


def blobs100(seed: int = 0) -> Workload:
    R = blob_set(100, 20.0, seed, 0, subs=(1, 2))
    S = blob_set(100, 20.0, seed, 1, subs=(1, 2))
    return Workload("blobs100", R, S, "within", taus=(0.5,))


def blobs20k(seed: int = 0, n: int = 20_000) -> Workload:
    side = scaled_side(400.0, 20_000, n)
    R = blob_set(n, side, seed, 0)
    S = blob_set(n, side, seed, 1)
    return Workload(f"blobs{n}", R, S, "within", taus=(0.0, 1.0))


def knn50k(seed: int = 0, n: int = 50_000, k: int = 3) -> Workload:
    side = 1000.0
    gmm = gmm_centres(seed, 20, side)
    R = blob_set(n, side, seed, 0, gmm=gmm)
    S = blob_set(n, side, seed, 1, gmm=gmm)
    return Workload(f"knn{n}", R, S, "knn", k=k)


def tubes2k(seed: int = 0, n_tubes: int = 2_000, n_blobs: int = 200_000) -> Workload:
    side = scaled_side(2320.0, 200_000, n_blobs)
    R = tube_set(n_tubes, side, seed, 0)
    S = blob_set(n_blobs, side, seed, 1)
    return Workload(f"tubes{n_tubes}x{n_blobs}", R, S, "within", taus=(2.0,))


STREAM_CHUNKS = 64


def stream2m_S(seed: int = 0, n_tubes: int = 20_000, side: float = 5000.0) -> MeshSet:
    return tube_set(n_tubes, side, seed, 1)


def stream2m_R_chunk(chunk: int, seed: int = 0, n: int = 2_000_000, chunks: int = STREAM_CHUNKS,
                     side: float = 5000.0) -> MeshSet:
    per = (n + chunks - 1) // chunks
    start = chunk * per
    count = max(0, min(n, start + per) - start)
    return blob_set(n, side, seed, 0, start=start, count=count)


def _tube_part(args):
    n, side, seed, set_id, start, count, lr = args
    return tube_set(n, side, seed, set_id, start=start, count=count, length_range=lr)


def tube_set_parallel(n: int, side: float, seed: int, set_id: int, procs: int = 16,
                      length_range=(50.0, 800.0)) -> MeshSet:
    """tube_set generated in ``procs`` spawned processes (same objects: each
    tube has its own random stream).  Start it before any CUDA call."""
    import multiprocessing as mp
    step = (n + procs - 1) // procs
    parts = [(n, side, seed, set_id, a, min(step, n - a), length_range) for a in range(0, n, step)]
    with mp.get_context("spawn").Pool(procs) as pool:
        return concat(pool.map(_tube_part, parts))


def _stream_chunk(args):
    return stream2m_R_chunk(*args)


def stream_chunks_parallel(chunks, procs: int = 16, seed: int = 0):
    """Chunks of the streamed workload's R, generated in spawned processes."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_stream_chunk, [(c, seed) for c in chunks])


def cadTI(seed: int = 0, t_models: int = 400, i_models: int = 100, replicas: int = 100,
          side: float = 1500.0) -> Workload:
    """CAD-like T x I join: t_models and i_models models, each replicated
    ``replicas`` times in a cube of side ``side``; intersection and within 1."""
    T = cad_set(t_models, replicas, side, seed, 0)
    I_ = cad_set(i_models, replicas, side, seed, 1)
    return Workload(f"cadTI{t_models}x{i_models}", T, I_, "within", taus=(0.0, 1.0))
