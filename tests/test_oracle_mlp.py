"""Pins of the MLP oracle (CPU only): finite-difference gradients, the BCE
closed form on a network reduced to a logistic regression, bfloat16 rounding
against hand-worked bit patterns, and an Adam step against its definition on a
one-parameter problem."""
import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    w = mlp.init_weights(3).astype(np.float64) + rng.normal(0, 0.05, mlp.N_PARAMS)
    X = rng.normal(size=(40, mlp.N_IN))
    y = (rng.random(40) < 0.4).astype(np.float64)
    loss, g = mlp.loss_and_grad(w, X, y)
    h = 1e-6
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [mlp.N_PARAMS - 1]])
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, X, y)[0] - mlp.loss_and_grad(wm, X, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), (i, fd, g[i])


def test_logistic_regression_special_case():
    """With a single active linear path the network is a logistic regression:
    loss = mean(log(1 + exp(-s z))) with s = +-1, gradient = X^T (sigmoid(z) - y) / n."""
    rng = np.random.default_rng(2)
    X = np.abs(rng.normal(size=(30, mlp.N_IN)))
    y = (rng.random(30) < 0.5).astype(np.float64)
    W1 = np.zeros((mlp.N_HID, mlp.N_IN))
    a = rng.normal(size=mlp.N_IN) * 0.3 + 1.0  # positive weights on positive inputs: ReLU passes
    W1[0] = a
    w2 = np.zeros(mlp.N_HID)
    w2[0] = 0.7
    w = mlp.pack(W1, np.zeros(mlp.N_HID), w2, -0.2)
    z = 0.7 * (X @ a) - 0.2
    ref = np.mean(np.where(y > 0, np.log1p(np.exp(-z)), np.log1p(np.exp(z))))
    loss, g = mlp.loss_and_grad(w, X, y)
    assert abs(loss - ref) < 1e-12
    p = 1 / (1 + np.exp(-z))
    assert np.allclose(mlp.unpack(g)[0][0], 0.7 * X.T @ (p - y) / 30, rtol=1e-12)
    assert abs(mlp.unpack(g)[3] - np.mean(p - y)) < 1e-12


def test_bf16_rounding_bit_patterns():
    # 1 + 2^-8 is exactly halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 3.0e38], dtype=np.float32)
    out = mlp.bf16_round(vals)
    want = [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, np.float64(np.float32(3.0e38).view(np.uint32) >> 16)]
    assert out[0] == want[0] and out[1] == want[1] and out[2] == want[2] and out[3] == want[3] and out[4] == want[4]
    assert out[5] > 2.9e38  # large values stay finite


def test_adam_step_definition():
    w, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    g = np.array([0.5])
    w1, m1, v1 = mlp.adam_step(w, m, v, g, 1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2, so w moves by lr * sign(g) (up to eps)
    assert abs(w1[0] - (1.0 - 0.1)) < 1e-7
    w2_, m2, v2 = mlp.adam_step(w1, m1, v1, g, 2, lr=0.1)
    mh = (0.9 * m1 + 0.1 * 0.5) / (1 - 0.9 ** 2)
    vh = (0.999 * v1 + 0.001 * 0.25) / (1 - 0.999 ** 2)
    assert abs(w2_[0] - (w1[0] - 0.1 * mh[0] / (np.sqrt(vh[0]) + 1e-8))) < 1e-12


def test_training_reduces_loss_on_separable_data():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(512, mlp.N_IN))
    y = (X[:, 0] + 0.5 * X[:, 3] > 0).astype(np.float64)
    w = mlp.init_weights(5).astype(np.float64)
    m, v = np.zeros_like(w), np.zeros_like(w)
    l0 = mlp.loss_and_grad(w, X, y)[0]
    for t in range(1, 301):
        _, g = mlp.loss_and_grad(w, X, y)
        w, m, v = mlp.adam_step(w, m, v, g, t, lr=1e-2)
    l1 = mlp.loss_and_grad(w, X, y)[0]
    assert l1 < 0.2 * l0
