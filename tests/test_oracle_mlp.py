"""Pins for the float64 MLP oracle: central finite differences, a closed-form
case and the Adam recurrence on a scalar."""
import math

import numpy as np

import oracle
from paper_2410_14088_gb300 import inputs


def params(seed, scale=0.3):
    return (inputs.uniform_array(seed, oracle.mlp_nparams()) - 0.5) * scale


def test_gradient_finite_differences():
    p = params(1)
    x = (inputs.uniform_array(2, 8 * 41) - 0.3).reshape(8, 41)
    t = inputs.uniform_array(3, 8)
    loss, g = oracle.mlp_loss_grad(p, x, t)
    rng_idx = (inputs.splitmix64_array(4, 64) % np.uint64(p.size)).astype(np.int64)
    h = 1e-6
    for i in rng_idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, x, t)[0] - oracle.mlp_loss_grad(pm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_closed_form_positive_path():
    # W1 = [I_41; 0], b1 = 0, W2 = I, b2 = 0, W3 = ones(64), b3 = 0.5, x >= 0:
    # ReLU passes everything, y = sum(x) + 0.5.
    n = oracle.mlp_nparams()
    p = np.zeros(n)
    W1 = np.zeros((64, 41)); W1[:41, :41] = np.eye(41)
    off = 0
    p[off:off + 64 * 41] = W1.ravel(); off += 64 * 41 + 64
    p[off:off + 64 * 64] = np.eye(64).ravel(); off += 64 * 64 + 64
    p[off:off + 64] = 1.0; off += 64
    p[off] = 0.5
    x = inputs.uniform_array(5, 3 * 41).reshape(3, 41)
    np.testing.assert_allclose(oracle.mlp_forward(p, x), x.sum(1) + 0.5, rtol=1e-14)
    # loss = mean 0.5 r^2, dL/db3 = mean r
    t = np.array([0.0, 1.0, 2.0])
    loss, g = oracle.mlp_loss_grad(p, x, t)
    r = x.sum(1) + 0.5 - t
    assert abs(loss - np.mean(0.5 * r * r)) < 1e-12
    assert abs(g[-1] - np.mean(r)) < 1e-12


def test_closed_form_relu_both_layers():
    # Layer 1 takes x and -x (first 23 inputs), so its ReLU gives relu(x_j) and relu(-x_j); layer 2 adds
    # the pair back to |x_j| on rows 0..22 and gives every other row the negated layer-1 unit minus 0.01,
    # a negative pre-activation that its ReLU must clear. With W3 = 1 on rows 0..22 and 2 elsewhere,
    # y = sum_{j<23} |x_j| + 0.25 only if both layers clamp at zero (no ReLU in layer 1 gives 0 for the
    # |x_j| rows; none in layer 2 adds the negative rows; a leaky or smooth activation shifts every term).
    n = oracle.mlp_nparams()
    W1 = np.zeros((64, 41))
    W1[:41, :41] = np.eye(41)
    W1[41:, :23] = -np.eye(23)
    W2 = np.zeros((64, 64))
    for j in range(23):
        W2[j, j] = W2[j, 41 + j] = 1.0
    for j in range(23, 64):
        W2[j, j] = -1.0
    b2 = np.zeros(64)
    b2[23:] = -0.01
    W3 = np.ones(64)
    W3[23:] = 2.0
    p = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), b2, W3, [0.25]])
    assert p.size == n
    x = (inputs.uniform_array(11, 4 * 41) - 0.5).reshape(4, 41)
    assert (x[:, :23] < 0).any() and (x[:, :23] > 0).any()
    y = oracle.mlp_forward(p, x)
    np.testing.assert_allclose(y, np.abs(x[:, :23]).sum(1) + 0.25, rtol=1e-14)
    # backward through the same ReLUs: rows with a negative pre-activation pass no gradient
    t = np.array([0.0, 1.0, 2.0, 3.0])
    loss, g = oracle.mlp_loss_grad(p, x, t)
    r = y - t
    o_b2, o_w3 = 64 * 41 + 64 + 64 * 64, 64 * 41 + 64 + 64 * 64 + 64
    np.testing.assert_allclose(g[o_b2:o_b2 + 23], np.full(23, r.mean()), rtol=1e-12)
    assert np.all(g[o_b2 + 23:o_b2 + 64] == 0.0)
    np.testing.assert_allclose(g[o_w3:o_w3 + 23], (r[:, None] * np.abs(x[:, :23])).mean(0), rtol=1e-12)
    assert np.all(g[o_w3 + 23:o_w3 + 64] == 0.0)


def test_adam_first_steps():
    # step 1: m = (1-b1) g, v = (1-b2) g^2, bias-corrected ratio = g/|g| -> p -= lr*sign(g)
    p = np.array([1.0, -2.0]); g = np.array([0.5, -3.0])
    m = np.zeros(2); v = np.zeros(2)
    oracle.adam_step(p, g, m, v, 1, lr=0.1, eps=0.0)
    np.testing.assert_allclose(p, [0.9, -1.9], rtol=1e-14)
    # step 2 with the same gradient: still exactly lr*sign(g)
    oracle.adam_step(p, g, m, v, 2, lr=0.1, eps=0.0)
    np.testing.assert_allclose(p, [0.8, -1.8], rtol=1e-13)
    np.testing.assert_allclose(m, 0.9 * 0.1 * g + 0.1 * g, rtol=1e-14)
