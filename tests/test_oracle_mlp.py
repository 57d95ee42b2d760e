"""Pins for the oracle's warm-start MLP: a hand-computed tiny network, a
central-difference gradient check, and the closed form of Adam's first step."""
import math

import numpy as np
import pytest

import oracle as O


def gelu(x):
    return 0.5 * x * (1 + math.erf(x / math.sqrt(2)))


def test_tiny_forward_by_hand():
    # 1 -> 1 (GELU) -> 1 linear
    sizes = [1, 1, 1]
    w1, b1, w2, b2 = 0.7, -0.2, 1.3, 0.05
    params = np.array([w1, b1, w2, b2])
    for x in (-1.5, 0.0, 0.4, 2.0):
        y = O.mlp_forward(sizes, params, np.array([[x]]))[0, 0]
        assert y == pytest.approx(w2 * gelu(w1 * x + b1) + b2, rel=1e-15, abs=1e-16)


def test_gradient_central_difference():
    sizes = [4, 8, 8, 6]
    rng = np.random.default_rng(3)
    n = O.mlp_param_count(sizes)
    p = rng.standard_normal(n) * 0.5
    x = rng.standard_normal((5, 4))
    t = rng.standard_normal((5, 6))
    loss, g = O.mlp_loss_grad(sizes, p, x, t)
    y = O.mlp_forward(sizes, p, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)
    h = 1e-6
    for i in rng.choice(n, 40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        num = (O.mlp_loss_grad(sizes, pp, x, t)[0] - O.mlp_loss_grad(sizes, pm, x, t)[0]) / (2 * h)
        assert g[i] == pytest.approx(num, rel=1e-6, abs=1e-9)


def test_adam_first_step_closed_form():
    # from zero moments, bias correction makes the first step lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    p = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    O.adam_step(p, m, v, g, lr=1e-2, t=1)
    assert np.allclose(p, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
