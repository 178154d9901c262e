"""Pins of the selector oracle (features, MLP backprop, AdamW, decision)
against closed forms and finite differences (no GPU)."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import selector_oracle as S


def test_param_count():
    assert S.NUM_PARAMS == 16 * 64 + 64 + 64 * 64 + 64 + 3 * 64 + 3


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.standard_normal(S.NUM_PARAMS) * 0.3
    X = rng.standard_normal((40, 16))
    y = rng.integers(0, 3, 40)
    w = np.array([1.0, 1.5, 2.5])
    _, g = S.loss_and_grad(theta, X, y, w)
    idx = rng.choice(S.NUM_PARAMS, 300, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        num = (S.loss_and_grad(theta + e, X, y, w)[0] - S.loss_and_grad(theta - e, X, y, w)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_features_of_graded_diagonal():
    n, kap = 32, 1e8
    d = kap ** (-np.arange(n) / (n - 1))
    f = S.features(np.diag(d), m=1 << 16)
    L = np.log10(d)
    assert f[0] == pytest.approx(8.0)
    assert f[1] == pytest.approx(-np.sort(L)[int(0.1 * 31)])
    assert f[2] == pytest.approx(-np.sort(L)[15])
    assert f[3] == pytest.approx(4.0)
    assert f[4] == pytest.approx(8.0 / 31 * math.sqrt((n * n - 1) / 12.0))
    assert 7.0 <= f[5] <= 8.0 + 1e-9          # power iteration underestimates both norms
    assert f[6] == pytest.approx(0.0, abs=1e-12)   # R D^-1 = I
    assert f[7] == pytest.approx(8.0)
    assert f[8] == 0.0
    assert f[9] == pytest.approx(32 / 512) and f[10] == pytest.approx(16 / 22)
    assert f[11] == pytest.approx(np.mean(d < 2.0 ** -11))
    assert f[12] == pytest.approx(np.mean(d < 2.0 ** -20))
    assert f[13] == pytest.approx(8.0)        # linear log-diagonal: slope -8/31
    assert f[14] == pytest.approx(8.0)
    assert f[15] == 1.0


def test_condition_estimate_bounds_true_condition():
    rng = np.random.default_rng(3)
    for kap in (1e2, 1e6, 1e10):
        n = 40
        Q1, _ = np.linalg.qr(rng.standard_normal((n, n)))
        Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
        A = Q1 @ np.diag(kap ** (-np.arange(n) / (n - 1))) @ Q2
        R = np.linalg.qr(A)[1]
        R = R * np.sign(np.diag(R))[:, None]
        f = S.features(R, m=4096)
        true = np.log10(np.linalg.cond(R))
        assert f[5] <= true + 1e-6 and f[5] >= true - 1.5


def test_cost_matrix_and_choice():
    C = S.cost_matrix([1.0, 1.02, 1.9])
    np.testing.assert_allclose(C, [[1.0, 2.02, 3.92], [1.02, 1.02, 2.92], [1.9, 1.9, 1.9]])
    theta = np.zeros(S.NUM_PARAMS)
    W1, b1, W2, b2, W3, b3 = S.unpack(theta)
    for k, expect in [(0, 0), (1, 1), (2, 2)]:
        t = theta.copy()
        t[-3:] = -50.0
        t[-3 + k] = 50.0            # b3 makes p = onehot(k)
        assert S.choose(t, np.zeros((1, 16)), [1.0, 1.02, 1.9])[0] == expect
    # uniform uncertainty between fp16 and fp64: the expected cost of fp64 wins
    t = theta.copy()
    t[-3:] = [0.0, -50.0, 0.0]
    assert S.choose(t, np.zeros((1, 16)), [1.0, 1.02, 1.9])[0] == 2


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(5).standard_normal(5000).astype(np.float32) * 7
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.round_bf16(x), ref)


def test_adamw_trains_separable_problem():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((600, 16))
    y = (X[:, 0] > 0.5).astype(int) + (X[:, 1] > 0.5).astype(int)
    theta = rng.standard_normal(S.NUM_PARAMS) * 0.1
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    w = np.ones(3)
    l0 = S.loss_and_grad(theta, X, y, w)[0]
    for step in range(1, 301):
        _, g = S.loss_and_grad(theta, X, y, w)
        theta, m, v = S.adamw_step(theta, g, m, v, step, lr=1e-2)
    l1 = S.loss_and_grad(theta, X, y, w)[0]
    acc = np.mean(np.argmax(S.forward(theta, X)[0], axis=1) == y)
    assert l1 < 0.3 * l0 and acc > 0.9
