"""The "zero_copy" context option: pj_load_set reads pinned host arrays in
place instead of staging them.  Sets loaded that way must give the same
join results bit for bit as sets loaded through the staging copies;
pageable arrays fall back to the copies."""
import copy

import numpy as np
import pytest

from synth import configs

pytestmark = pytest.mark.gpu


def pinned(ms):
    import torch
    out = copy.copy(ms)
    cache = {}

    def pin(a):
        if a is None:
            return None
        if id(a) not in cache:
            cache[id(a)] = torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        return cache[id(a)]

    for f in ("verts", "vert_off", "faces", "face_off", "hd", "ph"):
        setattr(out, f, [pin(a) for a in getattr(ms, f)])
    out.anchor = pin(ms.anchor)
    return out


def test_zero_copy_equals_staged():
    from paper_2604_19982_gb300 import pj
    w = configs.blobs20k(n=2000)
    Rp, Sp = pinned(w.R), pinned(w.S)
    ref = pj.Context(0)
    zc = pj.Context(0, {"zero_copy": 1})
    out = []
    for c, (R, S) in ((ref, (w.R, w.S)), (zc, (Rp, Sp)), (zc, (w.R, w.S))):
        gR, gS = c.load_set(R), c.load_set(S)
        res = [c.join(gR, gS, pj.WITHIN, tau=t, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST) for t in (0.0, 1.0)]
        res.append(c.join(gR, gS, pj.KNN, k=3, prec=pj.FP32, flags=pj.TILE_PRUNE | pj.EXACT_DIST))
        out.append(res)
        gR.free()
        gS.free()
    for res in out[1:]:
        for a, b in zip(res, out[0]):
            oa, ob = np.lexsort((a.s, a.r)), np.lexsort((b.s, b.r))
            for f in ("r", "s", "d_lo", "d_hi", "d", "exact"):
                assert np.array_equal(getattr(a, f)[oa], getattr(b, f)[ob]), f
    ref.close()
    zc.close()
