"""Pins of the FP64 reference network (oracle/mlp.py): central finite
differences of the loss, the linear special case (all units active) and
the zero-weight closed form."""
import numpy as np

from oracle import mlp


def test_gradients_by_finite_differences():
    rng = np.random.default_rng(0)
    W = mlp.init(3)
    W[1] = rng.normal(0, 0.3, 64)
    W[3] = rng.normal(0, 0.3, 64)
    W[5] = np.array([0.2])
    X = rng.normal(size=(40, 16))
    t = rng.normal(size=40)
    _, G = mlp.loss_and_grads(W, X, t)
    h = 1e-6
    for wi in range(6):
        flat = W[wi].reshape(-1)
        idx = rng.choice(flat.size, min(12, flat.size), replace=False)
        for j in idx:
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[wi].reshape(-1)[j] += h
            Wm[wi].reshape(-1)[j] -= h
            fd = (mlp.loss_and_grads(Wp, X, t)[0] - mlp.loss_and_grads(Wm, X, t)[0]) / (2 * h)
            assert abs(fd - G[wi].reshape(-1)[j]) <= 1e-6 * max(1.0, abs(fd)), (wi, j)


def test_linear_when_all_units_active():
    rng = np.random.default_rng(1)
    W = [np.abs(w) for w in mlp.init(5)]
    W[1] = np.abs(rng.normal(1, 0.1, 64))
    W[3] = np.abs(rng.normal(1, 0.1, 64))
    X = np.abs(rng.normal(size=(30, 16)))
    y, _ = mlp.forward(W, X)
    lin = (((X @ W[0].T + W[1]) @ W[2].T + W[3]) @ W[4]) + W[5][0]
    assert np.allclose(y, lin, rtol=1e-13, atol=1e-12)


def test_zero_weights_closed_form():
    W = [np.zeros(s) for s in mlp.SHAPES]
    W[5] = np.array([0.75])
    X = np.random.default_rng(2).normal(size=(10, 16))
    t = np.linspace(0, 1, 10)
    loss, G = mlp.loss_and_grads(W, X, t)
    assert np.isclose(loss, 0.5 * np.mean((0.75 - t) ** 2))
    assert np.isclose(G[5][0], np.mean(0.75 - t))
    assert all(np.all(g == 0) for g in G[:5])
