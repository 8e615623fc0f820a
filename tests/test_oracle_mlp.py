"""Pins of the surrogate network's FP64 oracle (CPU only): closed forms, brute
force on tiny networks and central finite differences for every gradient."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import mlp

SMALL = (8, 16, 12, 5)  # a tiny network of the same structure (three layers, GELU hidden)


def _rand_params(widths, seed, scale=0.5):
    r = np.random.default_rng(seed)
    p = r.uniform(-scale, scale, mlp.param_count(widths))
    # the padding columns of the first layer are zero, as the initialiser leaves them
    layers = mlp.unpack(p, widths)
    layers[0][0][:, widths[0]:] = 0.0
    return mlp.pack(layers)


def test_gelu_closed_forms():
    assert mlp.gelu(np.array(0.0)) == 0.0
    # GELU(x) = x Phi(x): Phi from scipy's normal CDF, not from erf
    for x in (-3.0, -1.0, 0.3, 1.0, 2.5):
        assert abs(mlp.gelu(np.array(x)) - x * stats.norm.cdf(x)) < 1e-15
    assert abs(mlp.gelu(np.array(12.0)) - 12.0) < 1e-12 and abs(mlp.gelu(np.array(-12.0))) < 1e-12
    assert abs(mlp.gelu_grad(np.array(0.0)) - 0.5) < 1e-15
    x = np.linspace(-4, 4, 81)
    h = 1e-5
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(x))) < 1e-9


def test_single_layer_is_an_affine_map():
    # no hidden layer: y = x W^T + b, summed by explicit loops
    widths = (8, 5)
    p = _rand_params(widths, 1)
    (W, b), = mlp.unpack(p, widths)
    x = np.random.default_rng(2).uniform(-1, 1, (7, 8))
    y, _ = mlp.forward(p, x, widths=widths)
    for r in range(7):
        for o in range(5):
            s = b[o]
            for i in range(8):
                s += W[o, i] * x[r, i]
            assert abs(y[r, o] - s) < 1e-14


def test_two_layer_forward_by_loops():
    widths = (8, 6, 3)
    p = _rand_params(widths, 3)
    (W1, b1), (W2, b2) = mlp.unpack(p, widths)
    x = np.random.default_rng(4).uniform(-1, 1, (5, 8))
    y, _ = mlp.forward(p, x, widths=widths)
    for r in range(5):
        h = [sum(W1[j, i] * x[r, i] for i in range(8)) + b1[j] for j in range(6)]
        h = [v * stats.norm.cdf(v) for v in h]
        for o in range(3):
            assert abs(y[r, o] - (sum(W2[o, j] * h[j] for j in range(6)) + b2[o])) < 1e-13


def test_parameter_and_input_gradients_by_finite_differences():
    p = _rand_params(SMALL, 5)
    r = np.random.default_rng(6)
    x = r.uniform(-1, 1, (4, 8))
    dy = r.standard_normal((4, SMALL[-1]))

    def L(pp, xx):
        return float(np.sum(dy * mlp.forward(pp, xx, widths=SMALL)[0]))

    _, cache = mlp.forward(p, x, widths=SMALL)
    gp, gx = mlp.backward(p, cache, dy, widths=SMALL)
    h = 1e-6
    idx = r.choice(p.size, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (L(p + e, x) - L(p - e, x)) / (2 * h)
        assert abs(fd - gp[i]) < 1e-6 * max(1.0, abs(fd)), i
    for rr in range(4):
        for c in range(8):
            e = np.zeros_like(x)
            e[rr, c] = h
            fd = (L(p, x + e) - L(p, x - e)) / (2 * h)
            assert abs(fd - gx[rr, c]) < 1e-6 * max(1.0, abs(fd))
    # padding columns of the first layer get no gradient (their inputs are 0)
    W1g = mlp.unpack(gp, SMALL)[0][0]
    assert np.all(W1g[:, 8:] == 0.0)


def test_deviance_minimiser_and_gradient():
    # argmin_y mean(y + S e^{-y}) = log mean(S): the network learns the log of the mean
    S = np.random.default_rng(7).exponential(2.5, size=(4000, 1))
    mu, sig = np.zeros(1), np.ones(1)
    ys = np.linspace(0.0, 2.0, 2001)
    losses = [mlp.deviance(np.full_like(S, y), S, mu, sig)[0] for y in ys]
    assert abs(ys[int(np.argmin(losses))] - math.log(S.mean())) < 2e-3
    # gradient by finite differences (with the standardisation y = mu + sigma y_hat)
    r = np.random.default_rng(8)
    yh = r.standard_normal((3, 6))
    S = r.exponential(1.0, (3, 6))
    mu, sig = r.uniform(-1, 1, 6), r.uniform(0.5, 2, 6)
    _, g = mlp.deviance(yh, S, mu, sig)
    h = 1e-6
    for i in range(3):
        for j in range(6):
            e = np.zeros_like(yh)
            e[i, j] = h
            fd = (mlp.deviance(yh + e, S, mu, sig)[0] - mlp.deviance(yh - e, S, mu, sig)[0]) / (2 * h)
            assert abs(fd - g[i, j]) < 1e-8


def test_design_loss_zero_at_target_and_gradient():
    r = np.random.default_rng(9)
    T = r.uniform(0.5, 3.0, (2, 10))
    mu, sig = r.uniform(-1, 1, 10), r.uniform(0.5, 2, 10)
    at = (np.log(T) - mu) / sig
    loss, g = mlp.design_loss(at, T, mu, sig)
    assert np.all(np.abs(loss) < 1e-20) and np.all(np.abs(g) < 1e-15)
    yh = at + 0.1 * r.standard_normal(at.shape)
    loss, g = mlp.design_loss(yh, T, mu, sig)
    assert np.all(g[:, 0] == 0.0)  # bin 0 (the squared mean) is left out
    h = 1e-6
    for i in range(2):
        for j in range(10):
            e = np.zeros_like(yh)
            e[i, j] = h
            fd = (mlp.design_loss(yh + e, T, mu, sig)[0][i] - mlp.design_loss(yh - e, T, mu, sig)[0][i]) / (2 * h)
            assert abs(fd - g[i, j]) < 1e-8


def test_adam_first_two_steps_closed_form():
    g1, g2 = np.array([0.3, -2.0, 1e-3]), np.array([-0.1, -1.0, 2e-3])
    p0 = np.array([1.0, -1.0, 0.5])
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    p1, m, v = mlp.adam(p0, np.zeros(3), np.zeros(3), g1, 1, lr, b1, b2, eps)
    # first step: m_hat = g, v_hat = g^2, so the update is lr g / (|g| + eps)
    np.testing.assert_allclose(p1, p0 - lr * g1 / (np.abs(g1) + eps), rtol=0, atol=1e-15)
    p2, _, _ = mlp.adam(p1, m, v, g2, 2, lr, b1, b2, eps)
    mh = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    np.testing.assert_allclose(p2, p1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-15)
    # decoupled weight decay adds lr wd p
    p1w, _, _ = mlp.adam(p0, np.zeros(3), np.zeros(3), g1, 1, lr, b1, b2, eps, wd=0.1)
    np.testing.assert_allclose(p1w, p1 - lr * 0.1 * p0, atol=1e-15)


def test_encode_decode_and_ranges():
    lo = np.array([[1.0, 0.5, 0.5, 0.0, 0.05, 0.01, 2.0, -1.0]])
    hi = np.array([[8.0, 2.0, 2.0, math.pi, 0.4, 0.1, 6.0, 1.0]])
    np.testing.assert_allclose(mlp.encode(lo), -np.ones((1, 8)), atol=1e-15)
    np.testing.assert_allclose(mlp.encode(hi), np.ones((1, 8)), atol=1e-15)
    t = np.random.default_rng(10).uniform(lo, hi, (50, 8))
    np.testing.assert_allclose(mlp.decode(mlp.encode(t)), t, rtol=1e-14, atol=1e-15)


def test_bf16_rounding():
    one = 1.0
    cases = {
        one: one,
        one + 2.0 ** -7: one + 2.0 ** -7,              # representable (8 significant bits)
        one + 2.0 ** -8: one,                          # halfway: ties to even (down)
        one + 3 * 2.0 ** -8: one + 2.0 ** -6,          # halfway: ties to even (up)
        one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7,  # above halfway
        -3.0: -3.0,
        0.0: 0.0,
    }
    for a, want in cases.items():
        assert mlp.bf16(np.array([a]))[0] == want, a
    x = np.random.default_rng(11).standard_normal(10000)
    rel = np.abs(mlp.bf16(x) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 + 1e-12


def test_init_ranges_and_uniformity():
    p = mlp.init(7)
    assert p.size == mlp.param_count() == 256 * 32 + 256 + 2 * (256 * 256 + 256) + 128 * 256 + 128
    layers = mlp.unpack(p)
    for l, (W, b) in enumerate(layers):
        fan = mlp.WIDTHS[l]
        assert np.all(b == 0.0)
        assert np.all(np.abs(W[:, :fan]) < 1.0 / math.sqrt(fan))
        if l == 0:
            assert np.all(W[:, fan:] == 0.0)
        u = W[:, :fan].reshape(-1) * math.sqrt(fan)
        assert stats.kstest(u, "uniform", args=(-1, 2)).pvalue > 1e-3
    assert not np.array_equal(p, mlp.init(8))
