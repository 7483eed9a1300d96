"""FP64 reference of the learned-proposal network and its training loss.

TEST INFRASTRUCTURE ONLY (see the package docstring).  A 24 -> 64 -> 64 -> 1
multilayer perceptron with ReLU, parameters packed as W1[64][24], b1[64],
W2[64][64], b2[64], w3[64], b3; logits s, targets t in [0, 1] (the plain
Metropolis acceptance of a logged candidate); loss = mean binary cross-entropy
of sigmoid(s) against t.  Written out with numpy matrix products only.
"""
from __future__ import annotations

import numpy as np

NPARAM = 64 * 24 + 64 + 64 * 64 + 64 + 64 + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    i = 0
    W1 = w[i:i + 64 * 24].reshape(64, 24); i += 64 * 24
    b1 = w[i:i + 64]; i += 64
    W2 = w[i:i + 64 * 64].reshape(64, 64); i += 64 * 64
    b2 = w[i:i + 64]; i += 64
    w3 = w[i:i + 64]; i += 64
    b3 = w[i]
    return W1, b1, W2, b2, w3, b3


def forward(w, F):
    """F: (B, 24) -> logits (B,), with the hidden activations."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    a1 = F @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3, (a1, h1, a2, h2)


def loss_and_grad(w, F, t):
    """Mean BCE of sigmoid(s) vs t and its gradient with respect to the packed parameters."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    s, (a1, h1, a2, h2) = forward(w, F)
    B = len(t)
    # log(1 + e^s) - t s, computed stably
    loss = np.mean(np.logaddexp(0.0, s) - t * s)
    ds = (1.0 / (1.0 + np.exp(-s)) - t) / B            # dL/ds
    g_w3 = h2.T @ ds
    g_b3 = ds.sum()
    d2 = np.outer(ds, w3) * (a2 > 0)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (a1 > 0)
    g_W1 = d1.T @ F
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def init(seed=0, scale=1.0):
    """He-style random initial parameters."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, scale * np.sqrt(2 / 24), (64, 24))
    W2 = rng.normal(0, scale * np.sqrt(2 / 64), (64, 64))
    w3 = rng.normal(0, scale * np.sqrt(1 / 64), 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]])
