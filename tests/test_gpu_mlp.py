"""The learned proposal's network on the tensor cores (bf16 operands, fp32
accumulation) against the FP64 reference network (oracle/mlp.py).

Tolerances: the forward pass is compared with the reference evaluated on
the same bf16-rounded inputs, weights and hidden activations (remaining
differences: fp32 accumulation order and rare bf16 rounding flips), within
2% of the output scale; gradients with un-rounded FP64 within 6% relative
(Frobenius norm) per tensor, the size of bf16 rounding of operands."""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2604_19982_gb300 import pj
    c = pj.Context(0)
    yield c
    c.close()


def bf16(x):
    """Round float64 values to bfloat16 (round to nearest even), back to float64."""
    f = np.asarray(x, np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(W, X):
    W1, b1, W2, b2, W3, b3 = [np.asarray(w, np.float64) for w in W]
    z1 = bf16(X) @ bf16(W1).T + b1
    h1 = bf16(np.maximum(z1, 0))
    z2 = h1 @ bf16(W2).T + b2
    return np.maximum(z2, 0) @ W3 + b3[0]


def weights(seed):
    rng = np.random.default_rng(seed)
    W = ref.init(seed)
    W[1] = rng.normal(0, 0.2, 64)
    W[3] = rng.normal(0, 0.2, 64)
    W[5] = np.array([0.1])
    return [np.asarray(w, np.float32) for w in W]


def features(n, seed):
    return np.random.default_rng(seed).normal(0, 1, (n, 16)).astype(np.float32)


def test_forward_matches_reference(ctx):
    import torch
    W = weights(1)
    ctx.mlp_set_weights(*W)
    X = features(3001, 2)
    dX = torch.from_numpy(X).cuda()
    out = torch.empty(len(X), dtype=torch.float32, device="cuda")
    ctx.mlp_forward(dX.data_ptr(), len(X), out.data_ptr())
    y = out.cpu().numpy().astype(np.float64)
    want = forward_bf16(W, X.astype(np.float64))
    scale = np.sqrt(np.mean(want ** 2))
    assert np.all(np.abs(y - want) <= 0.02 * (np.abs(want) + scale))
    y64, _ = ref.forward(W, X)
    assert np.sqrt(np.mean((y - y64) ** 2)) <= 0.05 * scale


def test_gradients_match_reference(ctx):
    import torch
    W = weights(3)
    ctx.mlp_set_weights(*W)
    X = features(2048, 4)
    t = np.random.default_rng(5).normal(0, 1, len(X)).astype(np.float32)
    dX = torch.from_numpy(X).cuda()
    dt = torch.from_numpy(t).cuda()
    shapes = ref.SHAPES
    G = [torch.zeros(int(np.prod(s)), dtype=torch.float32, device="cuda") for s in shapes]
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ctx.mlp_grad(dX.data_ptr(), dt.data_ptr(), len(X), loss.data_ptr(), [g.data_ptr() for g in G])
    torch.cuda.synchronize()
    want_loss, want = ref.loss_and_grads(W, X, t)
    assert abs(loss.item() - want_loss) <= 0.03 * want_loss
    for g, w, s in zip(G, want, shapes):
        g = g.cpu().numpy().reshape(s).astype(np.float64)
        assert np.linalg.norm(g - w) <= 0.06 * np.linalg.norm(w) + 1e-7, s


def test_training_reduces_loss_and_roundtrips(ctx, tmp_path):
    rng = np.random.default_rng(7)
    X = rng.normal(0, 1, (20000, 16)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.3 * np.abs(X[:, 3])).astype(np.float32)
    W0 = weights(8)
    ctx.mlp_set_weights(*W0)
    l0 = ref.loss_and_grads(W0, X, t)[0]
    ctx.mlp_train(X, t, epochs=25, seed=1)
    W1 = ctx.mlp_get_weights()
    l1 = ref.loss_and_grads(W1, X, t)[0]
    assert l1 < 0.2 * l0, (l0, l1)
    p = str(tmp_path / "w.bin")
    ctx.mlp_save(p)
    ctx.mlp_set_weights(*W0)
    ctx.mlp_load(p)
    for a, b in zip(ctx.mlp_get_weights(), W1):
        assert np.array_equal(a, b)


def test_pair_features(ctx):
    import torch
    from synth import configs
    w = configs.blobs100()
    gR, gS = ctx.load_set(w.R), ctx.load_set(w.S)
    rng = np.random.default_rng(0)
    pr = rng.integers(0, 100, 200).astype(np.int32)
    ps = rng.integers(0, 100, 200).astype(np.int32)
    out = torch.empty((200, 16), dtype=torch.float32, device="cuda")
    ctx.pair_features(gR, gS, pr, ps, out.data_ptr())
    f = out.cpu().numpy().astype(np.float64)
    a, b = w.R.mbb().astype(np.float64)[pr], w.S.mbb().astype(np.float64)[ps]
    gap = np.maximum(0, np.maximum(b[:, :3] - a[:, 3:], a[:, :3] - b[:, 3:]))
    md = np.sqrt((gap ** 2).sum(1))
    ad = np.linalg.norm(w.R.anchor[pr].astype(np.float64) - w.S.anchor[ps], axis=1)
    ca, cb = (a[:, :3] + a[:, 3:]) / 2, (b[:, :3] + b[:, 3:]) / 2
    assert np.allclose(f[:, 0], np.log1p(md), atol=1e-5)
    assert np.allclose(f[:, 1], np.log1p(ad), atol=1e-5)
    assert np.allclose(f[:, 2], np.log1p(np.linalg.norm(ca - cb, axis=1)), atol=1e-5)
    assert np.allclose(f[:, 10], np.log(w.R.n_faces(1, 0) + 1) / 10, atol=1e-6)
    assert np.allclose(f[:, 15], 1.0)
    hd0 = np.array([w.R.hd_of(0, r).max() for r in pr])
    assert np.allclose(f[:, 8], np.log1p(hd0), atol=1e-6)
    gR.free()
    gS.free()
