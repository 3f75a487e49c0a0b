"""FP64 oracle of the hit-ranking MLP (test infrastructure only).

A 2-layer perceptron, 12 features -> 64 ReLU units -> 1 logit, scores a
(candidate, compatible hit) pair; pairs with logit below a threshold are dropped
before the N-best selection.  Training minimises the mean binary cross-entropy
against truth labels with Adam.  The paper has no learned component; the
network, its features and its training are this project's learned-pruning
workload (12 features, 64 hidden units, bfloat16 weights).  Written as plain
matrix algebra in float64.

Parameter vector layout (897 values): W1[64][12] (row = hidden unit), b1[64],
w2[64], b2.  The forward pass of the GPU uses the weights rounded to bfloat16;
`bf16_round` gives the same rounding (to nearest, ties to even) so that the
oracle can evaluate with identical weights.
"""
from __future__ import annotations

import numpy as np

N_IN = 12
N_HID = 64
N_PARAMS = N_IN * N_HID + N_HID + N_HID + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    W1 = w[:N_IN * N_HID].reshape(N_HID, N_IN)
    b1 = w[N_IN * N_HID:N_IN * N_HID + N_HID]
    w2 = w[N_IN * N_HID + N_HID:N_IN * N_HID + 2 * N_HID]
    b2 = w[-1]
    return W1, b1, w2, b2


def pack(W1, b1, w2, b2):
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(w2), [float(b2)]])


def bf16_round(w):
    """float32 -> nearest bfloat16 (ties to even), returned as float64 values."""
    f = np.ascontiguousarray(w, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    out[nan] = np.nan
    return out


def forward(w, X):
    """Logits of feature rows X [n, 12]."""
    W1, b1, w2, b2 = unpack(w)
    A = np.asarray(X, dtype=np.float64) @ W1.T + b1
    H = np.maximum(A, 0.0)
    return H @ w2 + b2


def loss_and_grad(w, X, y):
    """Mean binary cross-entropy with logits and its gradient w.r.t. w."""
    W1, b1, w2, b2 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    A = X @ W1.T + b1
    H = np.maximum(A, 0.0)
    z = H @ w2 + b2
    # log(1 + exp(-|z|)) + max(z, 0) - z y
    loss = np.mean(np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z))))
    g = (1.0 / (1.0 + np.exp(-z)) - y) / n
    dw2 = H.T @ g
    db2 = g.sum()
    dA = np.outer(g, w2) * (A > 0)
    dW1 = dA.T @ X
    db1 = dA.sum(axis=0)
    return loss, pack(dW1, db1, dw2, db2)


def adam_step(w, m, v, g, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t is the 1-based step number); returns (w, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def init_weights(seed: int = 0):
    """He-normal first layer, small second layer, zero biases (float32 values)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((N_HID, N_IN)) * np.sqrt(2.0 / N_IN)
    w2 = rng.standard_normal(N_HID) * np.sqrt(1.0 / N_HID)
    return pack(W1, np.zeros(N_HID), w2, 0.0).astype(np.float32)
