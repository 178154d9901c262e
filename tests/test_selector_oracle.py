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


def test_adamw_first_step_closed_form():
    # Decoupled weight decay (Loshchilov & Hutter): on step 1 the bias
    # corrections turn m and v into g and g^2, so the update is exactly
    # lr (g / (|g| + eps) + wd theta).  A coupled decay (wd theta folded into g)
    # or a missing bias correction gives a different step.
    theta = np.array([0.5, -2.0, 3.0, 0.0])
    g = np.array([0.1, 0.3, -4.0, 1e-3])
    lr, wd, eps = 0.01, 0.1, 1e-8
    t1, m1, v1 = S.adamw_step(theta, g, np.zeros(4), np.zeros(4), 1, lr=lr, beta1=0.9, beta2=0.999, eps=eps, wd=wd)
    want = theta - lr * (g / (np.abs(g) + eps) + wd * theta)
    np.testing.assert_allclose(t1, want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)   # 1 - 0.999 rounds
    coupled = g + wd * theta
    t_coupled = theta - lr * coupled / (np.abs(coupled) + eps)
    assert np.abs(t1 - t_coupled).max() > 1e-4


def test_adamw_second_step_hand_computed():
    # step 2 by hand: m2 = b1 m1 + (1-b1) g2, v2 = b2 v1 + (1-b2) g2^2,
    # bias-corrected by 1 - b^2; theta3 = theta2 - lr (mh / (sqrt(vh) + eps) + wd theta2)
    b1, b2, lr, wd, eps = 0.9, 0.999, 0.05, 0.01, 1e-8
    th = np.array([1.0])
    g1, g2 = np.array([2.0]), np.array([-1.0])
    th1, m1, v1 = S.adamw_step(th, g1, np.zeros(1), np.zeros(1), 1, lr=lr, beta1=b1, beta2=b2, eps=eps, wd=wd)
    th2, _, _ = S.adamw_step(th1, g2, m1, v1, 2, lr=lr, beta1=b1, beta2=b2, eps=eps, wd=wd)
    # by hand: th1 = 1 - 0.05 (2/(2+1e-8) + 0.01) = 0.9495 (to 5e-10)
    assert abs(th1[0] - (1.0 - lr * (2.0 / (2.0 + eps) + wd))) < 1e-15
    m2 = 0.9 * 0.2 + 0.1 * (-1.0)                   # 0.08
    v2 = 0.999 * 0.004 + 0.001 * 1.0                # 0.004996
    mh, vh = m2 / (1 - 0.81), v2 / (1 - 0.998001)
    want = th1[0] - lr * (mh / (math.sqrt(vh) + eps) + wd * th1[0])
    assert abs(th2[0] - want) < 1e-15


def test_adamw_matches_torch_adamw_over_steps():
    # a library routine with the same definition: torch.optim.AdamW (decoupled
    # decay, bias correction), several steps with varying gradients, FP64
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    theta0 = rng.standard_normal(50)
    grads = rng.standard_normal((6, 50))
    lr, b1, b2, eps, wd = 3e-3, 0.9, 0.999, 1e-8, 1e-2
    p = torch.nn.Parameter(torch.from_numpy(theta0.copy()))
    opt = torch.optim.AdamW([p], lr=lr, betas=(b1, b2), eps=eps, weight_decay=wd)
    th, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads, start=1):
        p.grad = torch.from_numpy(g.copy())
        opt.step()
        th, m, v = S.adamw_step(th, g, m, v, k, lr=lr, beta1=b1, beta2=b2, eps=eps, wd=wd)
    np.testing.assert_allclose(th, p.detach().numpy(), rtol=0, atol=1e-14)


def test_mlp_loss_and_gradient_match_torch_autograd():
    # the same definitions in a library: logits of Linear(16, 64) -> ReLU -> Linear(64, 64) -> ReLU ->
    # Linear(64, 3) (weights stored out x in, bias after), the class-weighted cross-entropy summed over the
    # batch and divided by the batch size, and its gradient by torch's autograd, all in float64; a
    # transposed weight, a missing bias or ReLU, or a weight-normalised mean fails here
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(S.NUM_PARAMS) * 0.3
    X = rng.standard_normal((37, 16))
    y = rng.integers(0, 3, 37)
    w = np.array([1.0, 1.7, 3.0])
    loss, g = S.loss_and_grad(theta, X, y, w)
    z_or, _ = S.forward(theta, X)
    params = [torch.tensor(p, dtype=torch.float64, requires_grad=True) for p in S.unpack(theta.copy())]
    W1, b1, W2, b2, W3, b3 = params
    xt = torch.from_numpy(X)
    z = F.linear(F.relu(F.linear(F.relu(F.linear(xt, W1, b1)), W2, b2)), W3, b3)
    lt = F.cross_entropy(z, torch.from_numpy(y), weight=torch.from_numpy(w), reduction="sum") / X.shape[0]
    lt.backward()
    gt = np.concatenate([p.grad.numpy().ravel() for p in params])
    np.testing.assert_allclose(z_or, z.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert abs(loss - lt.item()) <= 1e-12 * abs(lt.item())
    np.testing.assert_allclose(g, gt, rtol=1e-10, atol=1e-13)
