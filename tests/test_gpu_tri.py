"""Triangle-distance kernels (pj_tri_dist) against the oracle.

FP64 kernel: equal to the oracle within 1e-12 relative (absolute floor
1e-14 for coordinates of order 1).  FP32 kernel: within the forward error
bound it reports.  Both: a distance is 0 exactly when the oracle's is
(the closed triangles meet), on every pair, including exact contacts and
one-float-step near misses.
"""
import numpy as np
import pytest

import oracle
from gpu_util import empty_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


def run(ctx, P, Q, prec):
    import torch
    from paper_2604_19982_gb300 import pj  # noqa: F401
    P32 = np.ascontiguousarray(P, np.float32).reshape(-1, 9)
    Q32 = np.ascontiguousarray(Q, np.float32).reshape(-1, 9)
    n = P32.shape[0]
    dP, dQ = to_dev(P32), to_dev(Q32)
    out = empty_dev(n, torch.float64)
    err = empty_dev(n, torch.float64)
    ctx.tri_dist(dP.data_ptr(), dQ.data_ptr(), n, prec, out.data_ptr(), err.data_ptr())
    torch.cuda.synchronize()
    return out.cpu().numpy(), err.cpu().numpy()


def random_pairs(rng, n, spread=3.0):
    P = rng.normal(size=(n, 3, 3)).astype(np.float32)
    Q = (rng.normal(size=(n, 3, 3)) + rng.normal(size=(n, 1, 3)) * rng.uniform(0, spread, (n, 1, 1))).astype(
        np.float32)
    return P, Q


def near_parallel_pairs(rng, n):
    """Edges at angles 1e-7..1e-1 rad, 1e-6..1 apart: the ill-conditioned
    regime of the segment-segment solve."""
    P = np.empty((n, 3, 3))
    Q = np.empty((n, 3, 3))
    for i in range(n):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        w = rng.normal(size=3)
        w -= (w @ u) * u
        w /= np.linalg.norm(w)
        v = np.cross(u, w)
        th = 10 ** rng.uniform(-7, -1)
        gap = 10 ** rng.uniform(-6, 0)
        L = rng.uniform(0.1, 2.0)
        c = rng.normal(size=3) * 5
        P[i, 0] = c
        P[i, 1] = c + L * u
        P[i, 2] = c + rng.uniform(0.1, 1) * u * L * 0.5 - rng.uniform(0.1, 1) * v
        du = np.cos(th) * u + np.sin(th) * w
        q0 = c + gap * v + rng.uniform(-0.5, 0.5) * L * u
        Q[i, 0] = q0
        Q[i, 1] = q0 + L * du
        Q[i, 2] = q0 + rng.uniform(0.1, 1) * L * 0.5 * du + rng.uniform(0.1, 1) * v
    return P.astype(np.float32), Q.astype(np.float32)


def test_fp64_random_matches_oracle(ctx):
    from paper_2604_19982_gb300 import pj
    rng = np.random.default_rng(1)
    P, Q = random_pairs(rng, 20000)
    d, _ = run(ctx, P, Q, pj.FP64)
    ref, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    assert np.array_equal(d == 0, ref == 0)
    assert (ref == 0).sum() > 100
    assert (np.abs(d - ref) <= 1e-12 * ref + 1e-14).all()


def test_fp64_closed_forms(ctx):
    from paper_2604_19982_gb300 import pj
    import test_oracle_pins as T
    cases = T._closed_forms()
    P = np.array([c[1] for c in cases])
    Q = np.array([c[2] for c in cases])
    want = np.array([c[3] for c in cases])
    for prec, tol in ((pj.FP64, 1e-14), (pj.FP32, 2e-6)):
        d, _ = run(ctx, P, Q, prec)
        d2, _ = run(ctx, Q, P, prec)
        assert np.allclose(d, want, rtol=0, atol=tol), (prec, d, want)
        assert np.allclose(d2, want, rtol=0, atol=tol)
    dp, _ = run(ctx, P, Q, pj.FP64)
    pierce = [c[0] for c in cases].index("pierce")
    assert dp[pierce] == 0.0


def test_fp32_within_reported_bound_random(ctx):
    from paper_2604_19982_gb300 import pj
    rng = np.random.default_rng(2)
    P, Q = random_pairs(rng, 200000)
    d, err = run(ctx, P, Q, pj.FP32)
    ref, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    assert (np.abs(d - ref) <= err).all()
    # typical single-precision error is far inside the worst-case bound,
    # whose 8 sqrt(u) L term covers nearly parallel edges
    assert np.median(np.abs(d - ref)) < 1e-5
    assert np.median(err) < 2e-2


def test_fp32_within_reported_bound_near_parallel(ctx):
    from paper_2604_19982_gb300 import pj
    rng = np.random.default_rng(3)
    P, Q = near_parallel_pairs(rng, 20000)
    d, err = run(ctx, P, Q, pj.FP32)
    ref, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    ratio = np.abs(d - ref) / err
    assert (ratio <= 1.0).all(), f"max |d32-d64|/bound = {ratio.max():.3f}"


def test_fp64_degenerate(ctx):
    from paper_2604_19982_gb300 import pj
    import test_oracle_pins as T
    rng = np.random.default_rng(11)
    P, Q = T._degenerate_pairs(rng)
    P = P.astype(np.float32)
    Q = Q.astype(np.float32)
    d, _ = run(ctx, P, Q, pj.FP64)
    ref, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    assert np.array_equal(d == 0, ref == 0)
    assert (np.abs(d - ref) <= 1e-12 * ref + 1e-12).all()


def piercing_pairs(rng, n):
    """Q's edge pierces P at depths 1e-7..1 (relative to the facet size
    0.1..10), away from P's edges, at offsets up to 1e3 from the origin: the
    crossing decisions go through the single-precision filter when clear and
    fall back to double precision when the depth is near the rounding."""
    P = np.empty((n, 3, 3))
    Q = np.empty((n, 3, 3))
    for i in range(n):
        L = 10 ** rng.uniform(-1, 1)
        c = rng.normal(size=3) * 10 ** rng.uniform(0, 3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        w = rng.normal(size=3)
        w -= (w @ u) * u
        w /= np.linalg.norm(w)
        nrm = np.cross(u, w)
        P[i] = [c, c + L * u, c + L * w]
        hit = c + L * (rng.uniform(0.2, 0.4) * u + rng.uniform(0.2, 0.4) * w)   # inside P
        depth = L * 10 ** rng.uniform(-7, 0)
        side = rng.normal(size=3) * 0.3
        a = hit + depth * nrm + side * depth
        b = hit - L * nrm * rng.uniform(0.3, 1.0)
        Q[i] = [a, b, b + L * (rng.normal(size=3) * 0.5)]
    return P.astype(np.float32), Q.astype(np.float32)


def check_zero_and_values(P, Q, ref, d64, d32, err):
    """Zero-ness equal to the oracle's on every pair (0 exactly when the
    closed triangles meet), non-zero distances within the tolerances:
    FP64 1e-12 relative above an absolute floor of a few u_64 times the
    coordinate scale (the candidate formulas differ in rounding), FP32
    within the bound the kernel reports."""
    zero = ref == 0
    assert np.array_equal(d64 == 0, zero), np.nonzero((d64 == 0) != zero)[0][:10]
    assert np.array_equal(d32 == 0, zero), np.nonzero((d32 == 0) != zero)[0][:10]
    nz = ~zero
    scale = np.maximum(np.abs(P.astype(np.float64)).reshape(len(P), -1).max(1),
                       np.abs(Q.astype(np.float64)).reshape(len(Q), -1).max(1))
    assert (np.abs(d64[nz] - ref[nz]) <= 1e-12 * ref[nz] + 1e-14 * scale[nz]).all()
    assert (np.abs(d32[nz] - ref[nz]) <= err[nz]).all()


def test_crossing_decisions_exact(ctx):
    """Piercing pairs at depths down to the rounding of the inputs: every
    pair's zero-ness equals the oracle's (exact meeting test on both sides:
    single-precision filtered signs, then exact arithmetic)."""
    from paper_2604_19982_gb300 import pj
    rng = np.random.default_rng(12)
    P, Q = piercing_pairs(rng, 20000)
    ref, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    d64, _ = run(ctx, P, Q, pj.FP64)
    d32, err = run(ctx, P, Q, pj.FP32)
    assert (ref == 0).sum() > 15000 and (ref > 0).sum() > 100
    check_zero_and_values(P, Q, ref, d64, d32, err)


@pytest.mark.parametrize("offset", [0.0, 1000.0])
def test_contacts_exact(ctx, offset):
    """Exact contacts of every kind (vertex on face, on edge, shared vertex,
    edge through edge, coplanar overlap, segment and point triangles) and
    one-float-step near misses: zero-ness equal to the oracle's on every
    pair, in both precisions."""
    from paper_2604_19982_gb300 import pj
    from meet_cases import contact_pairs
    rng = np.random.default_rng(41 if offset == 0 else 42)
    P, Q = contact_pairs(rng, 9000, offset)
    ref, _ = oracle.tri_dist(P.astype(np.float64), Q.astype(np.float64))
    d64, _ = run(ctx, P, Q, pj.FP64)
    d32, err = run(ctx, P, Q, pj.FP32)
    assert (ref == 0).sum() > 2000 and (ref > 0).sum() > 1000
    check_zero_and_values(P, Q, ref, d64, d32, err)
    # swapped roles give the same decisions
    e64, _ = run(ctx, Q, P, pj.FP64)
    assert np.array_equal(e64 == 0, ref == 0)
