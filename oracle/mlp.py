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


# ---------------------------------------------------------------------------
# The same network at the precision of a bf16 tensor-core implementation:
# inputs, W1, W2, the first hidden layer and the backward signals that enter
# products are rounded to bfloat16 (round to nearest, ties to even, directly
# from binary64); biases and w3 are binary32; everything else is exact (FP64)
# here.  Used where a bf16 network's outputs are compared.
# ---------------------------------------------------------------------------

def bf16(v):
    """Round to the nearest bfloat16 value (8 significant bits), ties to even."""
    v = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(v)
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def f32(v):
    return np.asarray(v, dtype=np.float32).astype(np.float64)


def unpack_bf16(w):
    W1, b1, W2, b2, w3, b3 = unpack(w)
    return bf16(W1), f32(b1), bf16(W2), f32(b2), f32(w3), float(f32(b3))


def forward_bf16(w, F):
    W1, b1, W2, b2, w3, b3 = unpack_bf16(w)
    Fb = bf16(F)
    a1 = Fb @ W1.T + b1
    h1 = bf16(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ w3 + b3, (Fb, a1, h1, a2, h2)


def loss_and_grad_bf16(w, F, t):
    """Mean BCE and its gradient with the bf16 network's rounding points."""
    W1, b1, W2, b2, w3, b3 = unpack_bf16(w)
    s, (Fb, a1, h1, a2, h2) = forward_bf16(w, F)
    B = len(t)
    loss = np.mean(np.logaddexp(0.0, s) - t * s)
    ds = (1.0 / (1.0 + np.exp(-s)) - t) / B
    g_w3 = h2.T @ ds
    g_b3 = ds.sum()
    d2 = np.outer(ds, w3) * (a2 > 0)
    g_b2 = d2.sum(axis=0)
    d2b = bf16(d2)
    g_W2 = d2b.T @ h1
    d1 = (d2b @ W2) * (a1 > 0)
    g_b1 = d1.sum(axis=0)
    g_W1 = bf16(d1).T @ Fb
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def sparse_dyadic(seed=0):
    """Weights for which a bf16/fp32 network computes the FP64 logits of bf16
    inputs exactly (up to binary32 rounding of short sums): hidden units 2j and
    2j+1 pass relu(+f_j) and relu(-f_j); the second layer and w3 hold a few
    powers of two per row.  Non-uniform proposals with reproducible decisions."""
    rng = np.random.default_rng(seed)
    W1 = np.zeros((64, 24))
    for j in range(24):
        W1[2 * j, j] = 1.0
        W1[2 * j + 1, j] = -1.0
    W2 = np.zeros((64, 64))
    for o in range(64):
        for i in rng.choice(48, 3, replace=False):
            W2[o, i] = rng.choice([-1.0, 1.0]) * 2.0 ** rng.integers(-2, 2)
    w3 = rng.choice([-1.0, 1.0], 64) * 2.0 ** rng.integers(-2, 1, 64)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]])
