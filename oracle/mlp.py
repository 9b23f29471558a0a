"""Plain FP64 reference of the learned proposal's network -- TEST
INFRASTRUCTURE (tests, smoke and the benchmark's CPU leg only).

A 16 -> 64 -> 64 -> 1 multilayer perceptron with ReLU after the two hidden
layers; trained to predict log(1 + d) of an object pair under the loss
L = mean over the batch of (y - t)^2 / 2.  Weights follow the library's
layout: W1 [64, 16], b1 [64], W2 [64, 64], b2 [64], W3 [64], b3 [1].
(The paper has no learned component; this network exists only to order the
k-NN refinement and pick a starting LoD, never to change a result.)
"""
from __future__ import annotations

import numpy as np

SHAPES = [(64, 16), (64,), (64, 64), (64,), (64,), (1,)]


def init(seed: int = 0):
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / 16), (64, 16))
    W2 = rng.normal(0, np.sqrt(2.0 / 64), (64, 64))
    W3 = rng.normal(0, np.sqrt(1.0 / 64), (64,))
    return [W1, np.zeros(64), W2, np.zeros(64), W3, np.zeros(1)]


def forward(W, X):
    """Outputs y [n] and the intermediate pre-activations (z1, z2) and
    activations (h1, h2)."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(w, np.float64) for w in W]
    X = np.asarray(X, np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3[0]
    return y, (z1, h1, z2, h2)


def loss_and_grads(W, X, t):
    """L = mean((y - t)^2) / 2 and its gradient w.r.t. every weight tensor
    (chain rule through the two ReLU layers)."""
    W1, b1, W2, b2, W3, b3 = [np.asarray(w, np.float64) for w in W]
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    y, (z1, h1, z2, h2) = forward(W, X)
    n = X.shape[0]
    r = y - t
    loss = 0.5 * np.mean(r * r)
    dy = r / n
    gW3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    dz2 = np.outer(dy, W3) * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]
