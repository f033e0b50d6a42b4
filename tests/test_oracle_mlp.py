"""Pins of the warm-start network oracle (oracle/mlp.py) against definitions that
do not go through its own code paths: GELU identities and values, the BF16
rounding of hand-picked binary32 patterns, back-propagation against central
finite differences of the loss, and the closed form of Adam's first step."""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import mlp


def test_gelu_identities_and_values():
    x = np.linspace(-6, 6, 97)
    # z Phi(z) - (-z) Phi(-z) = z (Phi(z) + Phi(-z) = 1)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, rtol=0, atol=1e-15)
    assert mlp.gelu(0.0) == 0.0
    assert abs(mlp.gelu(40.0) - 40.0) < 1e-12 and abs(mlp.gelu(-40.0)) < 1e-12
    # Phi(1) = 0.841344746068543 (tables), so GELU(1) = Phi(1)
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(mlp.gelu_grad(0.0) - 0.5) < 1e-16
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd, rtol=0, atol=1e-8)


def test_bf16_rounding_cases():
    cases = {
        1.0: 1.0,
        1.0 + 2.0 ** -8: 1.0,                        # tie -> even (mantissa 0)
        1.0 + 3 * 2.0 ** -8: 1.0 + 4 * 2.0 ** -8,    # tie -> even (mantissa 2)
        1.0 + 2.0 ** -8 + 2.0 ** -20: 1.0 + 2.0 ** -7,   # above the tie -> up
        -1.5: -1.5,                                   # representable
        1.0 + 2.0 ** -7 + 2.0 ** -9: 1.0 + 2.0 ** -7,    # below the half-way point -> down
        3.0e38: 1.765625 * 2.0 ** 127,               # 3e38 = 1.76323... 2^127
    }
    for a, want in cases.items():
        got = float(mlp.bf16_round(a))
        assert got == np.float32(want), (a, got, want)
    # idempotent, and exactly 8 significant bits
    x = np.random.default_rng(0).standard_normal(1000)
    r = mlp.bf16_round(x)
    np.testing.assert_array_equal(mlp.bf16_round(r), r)
    assert np.all((np.asarray(r, np.float32).view(np.uint32) & 0xFFFF) == 0)


def _small_net(sizes, seed=1):
    params = wl.mlp_init(sizes, seed)
    rng = np.random.default_rng(seed)
    params = [(W, rng.standard_normal(W.shape[0]) * 0.1) for W, _ in params]
    F = rng.standard_normal((7, sizes[0]))
    T = rng.standard_normal((7, sizes[-1]))
    return mlp.from_init(params, F, T), F, T


def test_backprop_matches_central_differences():
    net, F, T = _small_net((3, 5, 4, 2))
    X = (F - net.in_mean) / net.in_scale
    Ts = (T - net.out_mean) / net.out_scale
    _, gW, gb = mlp.loss_and_grads(net, X, Ts, rounding=False)
    h = 1e-6
    for l in range(3):
        for arr, g in ((net.W[l], gW[l]), (net.b[l], gb[l])):
            flat = arr.reshape(-1)
            for i in range(flat.size):
                old = flat[i]
                flat[i] = old + h
                lp = mlp.loss_and_grads(net, X, Ts, rounding=False)[0]
                flat[i] = old - h
                lm = mlp.loss_and_grads(net, X, Ts, rounding=False)[0]
                flat[i] = old
                assert abs((lp - lm) / (2 * h) - g.reshape(-1)[i]) < 1e-7, (l, i)


def test_rounded_forward_is_forward_of_rounded_weights():
    net, F, T = _small_net((4, 8, 8, 3))
    X = (F - net.in_mean) / net.in_scale
    a = mlp.forward(net, X, rounding=True)[-1][1]
    net.W = [mlp.bf16_round(W) for W in net.W]
    b = mlp.forward(net, X, rounding=False)[-1][1]
    np.testing.assert_array_equal(a, b)


def test_adam_first_step_closed_form():
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -4.0, 1e-3])]
    opt = mlp.Adam(lr=0.01)
    opt.step(p, g)
    # t = 1: m_hat = g, v_hat = g^2, step = lr g / (|g| + eps)
    want = np.array([1.0, -2.0, 3.0]) - 0.01 * g[0] / (np.abs(g[0]) + 1e-8)
    np.testing.assert_allclose(p[0], want, rtol=0, atol=1e-15)


def test_standardisation_and_features():
    mu = np.array([[1.0, math.e, 0.25], [math.e ** 2, 1.0, 0.75]])
    F = mlp.features(mu, P=2)
    np.testing.assert_allclose(F, [[0.0, 1.0, 0.25], [2.0, 0.0, 0.75]], atol=1e-15)
    fm, fs, tm, ts = mlp.standardisation(F, F[:, :1])
    np.testing.assert_allclose(fm, [1.0, 0.5, 0.5])
    np.testing.assert_allclose(fs, [1.0, 0.5, 0.25])


def test_training_fits_a_smooth_map():
    """Full-batch Adam on 256 pairs of a smooth 3 -> 2 map: the loss falls by 50x."""
    rng = np.random.default_rng(3)
    F = rng.uniform(-1, 1, (256, 3))
    T = np.stack([np.sin(F[:, 0]) + F[:, 1] * F[:, 2], np.cos(F[:, 1]) - 0.5 * F[:, 0]], axis=1)
    net = mlp.from_init(wl.mlp_init((3, 32, 32, 2), 2), F, T)
    hist = mlp.train(net, F, T, steps=300, lr=1e-2)
    assert hist[-1] < hist[0] / 50
