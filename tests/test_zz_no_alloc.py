"""pj_pair_bounds_static, the variant of pj_pair_bounds for callers that
may not allocate device memory (embedded in an application that owns every
device allocation, or unable to pay cudaMalloc's device-wide
synchronization): called through the C ABI twice in a row, its bounds must
equal those of pj_pair_bounds within the tolerance of the bounds tests.
Collected last so that a stop-at-first-failure run has run everything
else first; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

from synth import configs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2604_19982_gb300 import pj
    w = configs.blobs100()
    ctx = pj.Context(0)
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    rng = np.random.default_rng(12)
    pr = rng.integers(0, w.R.n, 300).astype(np.int32)
    ps = rng.integers(0, w.S.n, 300).astype(np.int32)
    yield pj, ctx, gR, gS, pr, ps
    ctx.close()


@pytest.mark.parametrize("lod", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_static_matches_allocating_entry_point(setup, lod, prec):
    import torch
    pj, ctx, gR, gS, pr, ps = setup
    want_lb, want_ub = ctx.pair_bounds(gR, gS, pr, ps, lod, prec)
    dpr = torch.from_numpy(pr).cuda()
    dps = torch.from_numpy(ps).cuda()
    n = len(pr)
    for call in range(2):
        lb = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        ub = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
        ctx.pair_bounds_static(gR, gS, dpr.data_ptr(), dps.data_ptr(), n, lod, prec, lb.data_ptr(), ub.data_ptr())
        torch.cuda.synchronize()
        got_lb, got_ub = lb.cpu().numpy(), ub.cpu().numpy()
        assert np.all(np.abs(got_lb - want_lb) <= 1e-12 * np.abs(want_lb) + 1e-14), f"call {call}"
        assert np.all(np.abs(got_ub - want_ub) <= 1e-12 * np.abs(want_ub) + 1e-14), f"call {call}"


def test_static_allocates_nothing():
    """On a fresh context whose workspace was never sized, two calls leave
    the library's allocation count and the context's workspace at what they
    were (a regression that took scratch from the workspace or allocated
    temporaries would change one of them)."""
    import torch
    from paper_2604_19982_gb300 import pj
    w = configs.blobs100()
    ctx = pj.Context(0)
    try:
        gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
        rng = np.random.default_rng(13)
        n = 200
        dpr = torch.from_numpy(rng.integers(0, w.R.n, n).astype(np.int32)).cuda()
        dps = torch.from_numpy(rng.integers(0, w.S.n, n).astype(np.int32)).cuda()
        lb = torch.empty(n, dtype=torch.float64, device="cuda")
        ub = torch.empty(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        before = ctx.stats()
        assert before["ws_bytes"] == 0
        for lod in (0, 1, 1):
            ctx.pair_bounds_static(gR, gS, dpr.data_ptr(), dps.data_ptr(), n, lod, 1, lb.data_ptr(), ub.data_ptr())
        after = ctx.stats()
        assert after["allocs"] == before["allocs"] and after["ws_bytes"] == 0
        assert np.isfinite(lb.cpu().numpy()).all()
    finally:
        ctx.close()


def test_static_rejects_bad_ids(setup):
    import torch
    pj, ctx, gR, gS, pr, ps = setup
    n = len(pr)
    bad = pr.copy()
    bad[n // 2] = gR.n              # one past the last object of R
    dpr = torch.from_numpy(bad).cuda()
    dps = torch.from_numpy(ps).cuda()
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pj.PJError) as e:
        ctx.pair_bounds_static(gR, gS, dpr.data_ptr(), dps.data_ptr(), n, 1, 0, out.data_ptr(), out.data_ptr())
    assert e.value.status == pj.PJ_EBOUNDS
    neg = ps.copy()
    neg[0] = -1
    dneg = torch.from_numpy(neg).cuda()
    with pytest.raises(pj.PJError) as e:
        ctx.pair_bounds_static(gR, gS, dps.data_ptr(), dneg.data_ptr(), n, 0, 1, out.data_ptr(), out.data_ptr())
    assert e.value.status == pj.PJ_EBOUNDS
    # the next good call is unaffected (the error word is cleared per call)
    good = torch.from_numpy(pr).cuda()
    ctx.pair_bounds_static(gR, gS, good.data_ptr(), dps.data_ptr(), n, 1, 0, out.data_ptr(), out.data_ptr())


def test_static_rejects_too_many_units(setup):
    """320-facet objects at full resolution: 10 x 10 blocks per pair, so 400
    pairs need up to 40,000 units, above PJ_STATIC_MAX_TILES (32,768)."""
    import torch
    pj, ctx, gR, gS, pr, ps = setup
    n = 400
    d = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(pj.PJError) as e:
        ctx.pair_bounds_static(gR, gS, d.data_ptr(), d.data_ptr(), n, 1, 0, out.data_ptr(), out.data_ptr())
    assert e.value.status == pj.PJ_EINVAL and "PJ_STATIC_MAX_TILES" in str(e.value)
    # at the coarse LoD (80 facets: 3 x 3 blocks) the same count fits
    ctx.pair_bounds_static(gR, gS, d.data_ptr(), d.data_ptr(), n, 0, 0, out.data_ptr(), out.data_ptr())


def test_static_rejects_oversize(setup):
    import torch
    pj, ctx, gR, gS, pr, ps = setup
    n = pj.lib().pj_pair_bounds_static  # noqa: F841 (symbol present)
    big = 4097
    dpr = torch.zeros(big, dtype=torch.int32, device="cuda")
    out = torch.zeros(big, dtype=torch.float64, device="cuda")
    with pytest.raises(pj.PJError) as e:
        ctx.pair_bounds_static(gR, gS, dpr.data_ptr(), dpr.data_ptr(), big, 1, 0, out.data_ptr(), out.data_ptr())
    assert e.value.status == pj.PJ_EINVAL and "PJ_STATIC_MAX_PAIRS" in str(e.value)
