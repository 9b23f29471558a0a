"""Voxels (section 2.1) and voxel-pair filtering (section 3.2, Algorithms 1
and 2) on the GPU against the voxel oracle, element by element: facet
labels at every LoD, k-means centres, voxel boxes and anchors, every voxel
pair's bounds, the object-pair bounds and decisions, and the surviving
voxel pairs in their order.  Both sides evaluate the same double-precision
expressions in the same order, so every comparison is exact.  The
single-precision filter (outward rounding) is checked against the same
oracle through the properties its rounding guarantees."""
import numpy as np
import pytest

from oracle import voxel as vx
from synth import configs
from gpu_util import empty_dev, to_dev
from voxel_cases import empty_and_two_triangles

pytestmark = pytest.mark.gpu

SETS = {
    "blobs_r": lambda: configs.blob_set(24, 30.0, 5, 0),
    "blobs_s": lambda: configs.blob_set(24, 30.0, 5, 1),
    "tubes": lambda: configs.tube_set(4, 60.0, 5, 2, length_range=(50.0, 120.0)),
    "empty": empty_and_two_triangles,
}


def _facets(ms, lod):
    return int(ms.face_off[lod][-1]) if ms.face_off[lod] is not None else ms.n * int(ms.faces[lod].shape[0])


@pytest.fixture(scope="module")
def env():
    from paper_2604_19982_gb300 import pj
    ctx = pj.Context(0, {"voxels": 1})
    ms = {k: f() for k, f in SETS.items()}
    g = {k: ctx.load_set(m) for k, m in ms.items()}
    ov = {k: vx.voxelize_set(m) for k, m in ms.items()}
    yield ctx, ms, g, ov
    ctx.close()


@pytest.mark.parametrize("kind", list(SETS))
def test_voxels_equal_oracle(env, kind):
    ctx, ms, g, ov = env
    m, o = ms[kind], ov[kind]
    got = ctx.voxels(g[kind])
    want_off = np.concatenate([[0], np.cumsum([v["centres"].shape[0] for v in o])])
    assert np.array_equal(got["voxel_off"], want_off)
    assert ctx.voxel_count(g[kind]) == want_off[-1]
    cat = (lambda key, w: np.concatenate([v[key] for v in o]) if want_off[-1] else np.zeros((0, w)))
    assert np.array_equal(got["centres"], cat("centres", 3))
    assert np.array_equal(got["boxes"].astype(np.float64), cat("boxes", 6))
    assert np.array_equal(got["anchors"].astype(np.float64), cat("anchors", 3), equal_nan=True)
    for lod in range(m.n_lods):
        lab = ctx.voxel_labels(g[kind], lod, _facets(m, lod))
        want = np.concatenate([v["labels"][lod] for v in o])
        assert np.array_equal(lab, want), f"LoD {lod}: {(lab != want).sum()} labels differ"


def _mbb(ms):
    out = np.empty((ms.n, 6))
    for o in range(ms.n):
        v = ms.object_verts(ms.n_lods - 1, o).astype(np.float64)
        out[o, :3] = v.min(0) if v.size else np.inf
        out[o, 3:] = v.max(0) if v.size else -np.inf
    return out


def _pairs(mr, ms_, near, n_far, seed):
    """Pairs whose object boxes lie within `near`, plus n_far random others."""
    a, b = _mbb(mr), _mbb(ms_)
    g = np.maximum(0.0, np.maximum(b[None, :, :3] - a[:, None, 3:], a[:, None, :3] - b[None, :, 3:]))
    d = np.sqrt((g * g).sum(2))
    r, s = np.nonzero(d <= near)
    rng = np.random.default_rng(seed)
    fr = rng.integers(0, mr.n, n_far)
    fs = rng.integers(0, ms_.n, n_far)
    return np.concatenate([r, fr]).astype(np.int32), np.concatenate([s, fs]).astype(np.int32)


def _run(ctx, gR, gS, pr, ps, tau, cap, prec=0):
    import torch
    n = len(pr)
    out = {
        "op_lb": empty_dev(n, torch.float64), "op_ub": empty_dev(n, torch.float64),
        "status": empty_dev(n, torch.uint8), "vp_off": empty_dev(n + 1, torch.int64),
        "vp_lb": empty_dev(max(cap, 1), torch.float64), "vp_ub": empty_dev(max(cap, 1), torch.float64),
        "kept_off": empty_dev(n + 1, torch.int64), "kept": empty_dev(2 * max(cap, 1), torch.int32),
    }
    dpr, dps = to_dev(pr), to_dev(ps)
    nk = ctx.voxel_filter(gR, gS, dpr.data_ptr(), dps.data_ptr(), n, tau, {k: v.data_ptr() for k, v in out.items()},
                          cap, prec=prec)
    torch.cuda.synchronize()
    h = {k: v.cpu().numpy() for k, v in out.items()}
    h["kept"] = h["kept"][:2 * nk].reshape(-1, 2)
    tot = int(h["vp_off"][-1])
    h["vp_lb"] = h["vp_lb"][:tot]
    h["vp_ub"] = h["vp_ub"][:tot]
    return nk, h


CASES = [("blobs_r", "blobs_s", 3.0, 20), ("tubes", "blobs_s", 6.0, 10), ("blobs_r", "blobs_r", 2.0, 8),
         ("empty", "empty", 10.0, 0)]


@pytest.mark.parametrize("case", CASES, ids=[f"{a}-{b}" for a, b, _, _ in CASES])
@pytest.mark.parametrize("tau", [-1.0, 0.0, 0.5, 2.0])
def test_filter_equals_oracle(env, case, tau):
    ctx, ms, g, ov = env
    kr, ks, near, n_far = case
    if kr == "empty":
        pr = np.array([0, 1, 0, 1], np.int32)
        ps = np.array([1, 1, 0, 0], np.int32)
    else:
        pr, ps = _pairs(ms[kr], ms[ks], near, n_far, 7)
    want = vx.voxel_filter(ov[kr], ov[ks], pr, ps, tau)
    cap = int(want["vp_off"][-1])
    nk, got = _run(ctx, g[kr], g[ks], pr, ps, tau, cap)
    for key in ("vp_off", "op_lb", "op_ub", "status", "vp_lb", "vp_ub", "kept_off"):
        assert np.array_equal(got[key], want[key]), key
    assert nk == want["kept"].shape[0]
    assert np.array_equal(got["kept"], want["kept"])
    if kr != "empty" and tau < 0:
        assert 0 < nk < cap     # the pruning keeps some voxel pairs and drops others


REL32 = 4e-6     # single-precision bounds: a few roundings of 2^-24 each, outward


def _near(x, y):
    """x within REL32 (relative) of y."""
    return abs(x - y) <= REL32 * max(abs(x), abs(y))


@pytest.mark.parametrize("case", CASES, ids=[f"{a}-{b}" for a, b, _, _ in CASES])
@pytest.mark.parametrize("tau", [-1.0, 0.5, 2.0])
def test_filter_fp32_bounds_are_outward(env, case, tau):
    """Single precision rounded outward: every lower bound at most the exact
    (oracle) one and every upper bound at least it, each within REL32; the
    decisions equal the oracle's except within rounding of tau; the
    survivors contain the oracle's, and any extra voxel pair lies within
    rounding of the pair's upper bound."""
    from paper_2604_19982_gb300 import pj
    ctx, ms, g, ov = env
    kr, ks, near, n_far = case
    if kr == "empty":
        pr = np.array([0, 1, 0, 1], np.int32)
        ps = np.array([1, 1, 0, 0], np.int32)
    else:
        pr, ps = _pairs(ms[kr], ms[ks], near, n_far, 7)
    want = vx.voxel_filter(ov[kr], ov[ks], pr, ps, tau)
    cap = int(want["vp_off"][-1])
    nk, got = _run(ctx, g[kr], g[ks], pr, ps, tau, cap, prec=pj.FP32)
    assert np.array_equal(got["vp_off"], want["vp_off"])
    tiny = 1e-15
    for lo_key, hi_key in (("vp_lb", "vp_ub"), ("op_lb", "op_ub")):
        for key, lower in ((lo_key, True), (hi_key, False)):
            a, b = got[key], want[key]
            fin = np.isfinite(b)
            assert np.array_equal(np.isfinite(a), fin), key
            a, b = a[fin], b[fin]
            if lower:
                assert (a <= b * (1 + tiny)).all() and (a >= b * (1 - REL32)).all(), key
            else:
                assert (a >= b * (1 - tiny)).all() and (a <= b * (1 + REL32)).all(), key
    for p in range(len(pr)):
        gs, ws = int(got["status"][p]), int(want["status"][p])
        if gs != ws:
            # only where the deciding bound lies within rounding of tau
            assert _near(want["op_ub"][p], tau) or _near(want["op_lb"][p], tau), (p, gs, ws)
        gk = [tuple(x) for x in got["kept"][got["kept_off"][p]:got["kept_off"][p + 1]].tolist()]
        wk = [tuple(x) for x in want["kept"][want["kept_off"][p]:want["kept_off"][p + 1]].tolist()]
        assert gk == sorted(gk) and len(set(gk)) == len(gk)
        if gs == 0 and ws == 0:
            assert set(wk) <= set(gk)
        if gs != 0:
            assert gk == []
        ns = int(want["vp_off"][p + 1] - want["vp_off"][p]) // max(1, ov[kr][pr[p]]["centres"].shape[0])
        oub = want["op_ub"][p]
        for i, j in set(gk) - set(wk):
            lb = want["vp_lb"][want["vp_off"][p] + i * ns + j]
            assert lb <= oub * (1 + 3 * REL32), (p, i, j)


def test_filter_sizes_and_errors(env):
    from paper_2604_19982_gb300 import pj
    ctx, ms, g, ov = env
    pr = np.array([0, 1, 2], np.int32)
    ps = np.array([3, 4, 5], np.int32)
    want = vx.voxel_filter(ov["blobs_r"], ov["blobs_s"], pr, ps, -1.0)
    cap = int(want["vp_off"][-1])
    with pytest.raises(pj.PJError) as e:
        _run(ctx, g["blobs_r"], g["blobs_s"], pr, ps, -1.0, cap - 1)
    assert e.value.status == pj.PJ_EINVAL
    bad = np.array([0, 24, 2], np.int32)
    with pytest.raises(pj.PJError) as e:
        _run(ctx, g["blobs_r"], g["blobs_s"], bad, ps, -1.0, 10 * cap)
    assert e.value.status == pj.PJ_EBOUNDS
    with pytest.raises(pj.PJError) as e:
        _run(ctx, g["blobs_r"], g["blobs_s"], pr, ps, -1.0, cap, prec=7)
    assert e.value.status == pj.PJ_EINVAL
    nk, got = _run(ctx, g["blobs_r"], g["blobs_s"], pr[:0], ps[:0], -1.0, 0)
    assert nk == 0 and got["vp_off"][0] == 0 and got["kept_off"][0] == 0
    # a larger capacity than needed changes nothing
    nk, got = _run(ctx, g["blobs_r"], g["blobs_s"], pr, ps, -1.0, cap + 100)
    assert np.array_equal(got["kept"], want["kept"])
    st = ctx.stats()
    assert st["op_pairs"] == 3 and st["voxel_pairs"] == cap and st["kept"] == nk


def test_set_without_voxels_is_rejected(env):
    from paper_2604_19982_gb300 import pj
    _, ms, _, _ = env
    ctx = pj.Context(0)
    try:
        gs = ctx.load_set(ms["blobs_r"])
        with pytest.raises(pj.PJError) as e:
            ctx.voxel_count(gs)
        assert e.value.status == pj.PJ_EINVAL
        with pytest.raises(pj.PJError) as e:
            _run(ctx, gs, gs, np.array([0], np.int32), np.array([1], np.int32), -1.0, 10000)
        assert e.value.status == pj.PJ_EINVAL
    finally:
        ctx.close()


def test_voxel_partition_is_shared_by_the_joins_results(env):
    # loading with voxels changes no join result
    from paper_2604_19982_gb300 import pj
    ctx, ms, g, _ = env
    plain = pj.Context(0)
    try:
        a = ctx.join(g["blobs_r"], g["blobs_s"], pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
        pR, pS = plain.load_set(ms["blobs_r"]), plain.load_set(ms["blobs_s"])
        b = plain.join(pR, pS, pj.WITHIN, tau=1.0, prec=pj.FP32, flags=pj.TILE_PRUNE)
        assert np.array_equal(a.r, b.r) and np.array_equal(a.s, b.s)
    finally:
        plain.close()
