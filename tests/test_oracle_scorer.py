"""Pins for the scorer oracle: finite differences, the logistic-regression special
case, Adam's first step, BCE and GELU closed forms, BF16 rounding."""
import math

import numpy as np
import pytest
import torch
from scipy.stats import norm

from oracle import scorer as S


def test_gelu_matches_x_phi():
    x = np.linspace(-6, 6, 101)
    assert np.allclose(S.gelu(x), x * norm.cdf(x), atol=1e-14)
    h = 1e-6
    fd = (S.gelu(x + h) - S.gelu(x - h)) / (2 * h)
    assert np.allclose(S.gelu_grad(x), fd, atol=1e-8)


def test_bce_closed_form():
    assert S.bce(np.zeros(4), np.array([0, 1, 0, 1.0])) == pytest.approx(math.log(2), rel=1e-15)
    z = np.array([30.0, -30.0])
    assert S.bce(z, np.array([1.0, 0.0])) == pytest.approx(math.log1p(math.exp(-30)), rel=1e-12)


def test_logistic_regression_special_case():
    # with no hidden layer the network is logistic regression: dL/dw = X^T (sigma(Xw+b) - y) / B
    layers = (7, 1)
    g = np.random.default_rng(0)
    X = g.normal(size=(11, 7))
    y = (g.uniform(size=11) < 0.5).astype(float)
    theta = g.normal(size=S.n_params(layers))
    w, b = theta[:7], theta[7]
    p = 1.0 / (1.0 + np.exp(-(X @ w + b)))
    grad, loss = S.backward(theta, X, y, layers)
    assert np.allclose(grad[:7], X.T @ (p - y) / 11, atol=1e-14)
    assert grad[7] == pytest.approx(np.mean(p - y), abs=1e-14)
    assert loss == pytest.approx(np.mean(-y * np.log(p) - (1 - y) * np.log(1 - p)), rel=1e-12)


@pytest.mark.parametrize("layers", [(6, 5, 4, 1), (20, 8, 3, 1)])
def test_gradient_finite_differences(layers):
    g = np.random.default_rng(sum(layers))
    X = g.normal(size=(9, layers[0]))
    y = (g.uniform(size=9) < 0.5).astype(float)
    theta = g.normal(size=S.n_params(layers)) * 0.5
    grad, _ = S.backward(theta, X, y, layers)
    h = 1e-6
    for i in g.choice(theta.size, size=min(40, theta.size), replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (S.bce(S.forward(tp, X, layers)[0], y) - S.bce(S.forward(tm, X, layers)[0], y)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-7 + 1e-6 * abs(fd)


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    theta, m, v = S.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 1e-2)
    assert np.allclose(theta, -1e-2 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_round_matches_torch():
    x = np.random.default_rng(1).normal(size=1000).astype(np.float32) * 10
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(S.bf16_round(x), ref)


def test_cutout_brute_force_and_edges():
    g = np.random.default_rng(2)
    zp = g.normal(size=(100, 9, 9))
    bounds = [(0, 40), (40, 100)]
    trig = [(45, 4, 4), (2, 0, 8), (39, 8, 0)]
    cut = S.cutouts(zp, bounds, trig).reshape(3, 64, 5, 5)
    # interior: channels 13..76 clipped to coarse channel 1 (40..99), pixels 2..6
    assert np.array_equal(cut[0, 64 - 32 + 40 - 45:, :, :][:0].ravel(), np.array([]))
    assert np.array_equal(cut[0, 27:59], zp[40:72, 2:7, 2:7])
    assert not cut[0, :27].any()
    # corner trigger: rows/cols outside the image are zero, channels clipped to 0..39
    assert np.array_equal(cut[1, 30:64, 2:, :3], zp[0:34, 0:3, 6:9])
    assert not cut[1, :30].any() and not cut[1, :, :2].any() and not cut[1, :, :, 3:].any()
    assert np.array_equal(cut[2, :33, :3, 2:], zp[7:40, 6:9, 0:3]) and not cut[2, 33:].any()
