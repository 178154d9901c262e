"""Selector kernels (features, BF16 MLP forward/backward, AdamW, AUTO path)
against the FP64 selector oracle on the same (BF16-rounded) weights."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from oracle import selector_oracle as SO
from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_18411_gb300 import build
    build.build()
    from paper_2606_18411_gb300 import mrcqr as M
    from paper_2606_18411_gb300 import selector as S
    return torch, M, S


@pytest.mark.parametrize("m,n,kappa,kind", [(8192, 32, 1e2, "geometric"), (16384, 100, 1e10, "cliff"),
                                            (20000, 256, 1e14, "loguniform"), (4096, 17, 1e6, "clustered")])
def test_features_match_oracle(env, m, n, kappa, kind):
    torch, M, S = env
    A = M.to_colmajor(inputs.make_matrix(m, n, kappa, kind=kind, seed=n))
    Y = M.sketch(A, 2 * n, "fp16", seed=1)
    Rs = M.sketch_qr(Y, "fp16")
    f = torch.empty(16, dtype=torch.float32, device="cuda")
    from paper_2606_18411_gb300 import _lib
    assert _lib.load().mrcqr_selector_features(m, n, Rs.data_ptr(), f.data_ptr(),
                                               torch.cuda.current_stream().cuda_stream) == 0
    ref = SO.features(Rs.cpu().numpy(), m)
    np.testing.assert_allclose(f.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)


def _rand_setup(torch, S, B=300, seed=0):
    rng = np.random.default_rng(seed)
    theta = (rng.standard_normal(SO.NUM_PARAMS) * 0.3).astype(np.float32)
    X = (rng.standard_normal((B, 16)) * 3 + 1).astype(np.float32)
    y = rng.integers(0, 3, B).astype(np.int32)
    mu = X.mean(0)
    sd = X.std(0)
    return theta, X, y, mu, sd


def test_forward_and_gradient_match_oracle(env):
    torch, M, S = env
    theta, X, y, mu, sd = _rand_setup(torch, S)
    tr = S.Trainer(theta, mu, sd)
    theta_b = SO.round_bf16(theta)                       # the weights the kernels use
    Xn = (X.astype(np.float64) - mu) / sd
    Xd = torch.from_numpy(X).cuda()
    logits, choice = tr.forward(Xd, [1.0, 1.02, 1.9])
    z_ref, _ = SO.forward(theta_b, Xn)
    np.testing.assert_allclose(logits.cpu().numpy(), z_ref, rtol=1e-4, atol=1e-4)
    np.testing.assert_array_equal(choice.cpu().numpy(), SO.choose(theta_b, Xn, [1.0, 1.02, 1.9]))
    cw = np.array([1.0, 1.5, 2.5], np.float32)
    g = torch.zeros(SO.NUM_PARAMS, dtype=torch.float32, device="cuda")
    loss = tr.train_step(Xd, torch.from_numpy(y).cuda(), torch.from_numpy(cw).cuda(), apply=False, grad_out=g)
    l_ref, g_ref = SO.loss_and_grad(theta_b, Xn, y, cw.astype(np.float64))
    assert abs(float(loss.item()) - l_ref) <= 1e-5 * l_ref
    gh = g.cpu().numpy()
    for part, ref in zip(SO.unpack(gh.astype(np.float64)), SO.unpack(g_ref)):
        assert np.linalg.norm(part - ref) <= 1e-4 * np.linalg.norm(ref) + 1e-9


def test_adamw_step_matches_oracle(env):
    torch, M, S = env
    theta, X, y, mu, sd = _rand_setup(torch, S, seed=1)
    tr = S.Trainer(theta, mu, sd)
    cw = torch.ones(3, dtype=torch.float32, device="cuda")
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    g = torch.zeros(SO.NUM_PARAMS, dtype=torch.float32, device="cuda")
    tr.train_step(Xd, yd, cw, lr=1e-2, apply=False, grad_out=g)
    tr.train_step(Xd, yd, cw, lr=1e-2, apply=True)
    ref, _, _ = SO.adamw_step(theta.astype(np.float64), g.cpu().numpy().astype(np.float64),
                              np.zeros(SO.NUM_PARAMS), np.zeros(SO.NUM_PARAMS), 1, lr=1e-2)
    np.testing.assert_allclose(tr.master.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(tr.wbf16.view(torch.bfloat16).float().cpu().numpy(),
                                  SO.round_bf16(tr.master.cpu().numpy()))


def test_training_on_gpu_reduces_loss(env):
    torch, M, S = env
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2000, 16)).astype(np.float32)
    y = ((X[:, 0] > 0.3).astype(int) + (X[:, 3] > 0.3).astype(int)).astype(np.int32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    tr, mu, sd, losses = S.train(Xd, yd, epochs=25, batch=200, lr=1e-2)
    assert losses[-1] < 0.35 * losses[0]
    logits, _ = tr.forward(Xd, [1.0, 1.0, 1.0])
    assert np.mean(np.argmax(logits.cpu().numpy(), axis=1) == y) > 0.9


@pytest.mark.parametrize("forced", [0, 1, 2])
def test_auto_path_follows_selector_choice(env, forced):
    torch, M, S = env
    # weights whose output bias forces the class `forced`
    theta = np.zeros(SO.NUM_PARAMS, np.float32)
    theta[-3:] = -40.0
    theta[-3 + forced] = 40.0
    mu, sd, costs = np.zeros(16, np.float32), np.ones(16, np.float32), np.array([1, 1.02, 1.9], np.float32)
    S.set_weights(theta, mu, sd, costs)
    A = inputs.make_matrix(8192, 48, 1e6, seed=44)
    Q, R = M.factor(M.to_colmajor(A), prec="auto", seed=2)
    st = M.last_status()
    assert st["status"] == "OK" and st["selector_choice"] == forced
    assert st["prec_first"] == ["fp16", "fp32", "fp64"][forced]
    # kappa = 1e6: fp16 fails and escalates to fp32; fp32 / fp64 pass at once
    assert st["prec_used"] == ("fp32" if forced == 0 else ["fp16", "fp32", "fp64"][forced])
    assert O.orthogonality_error(Q.cpu().numpy())[0] <= 1e-13
    assert O.residual_error(A, Q.cpu().numpy(), R.cpu().numpy())[0] <= 1e-13


def _shipped_costs(S):
    """Relative run costs fp16 / fp32 / fp64 stored in the shipped weights file."""
    with open(S.DEFAULT_WEIGHTS, "rb") as f:
        b = f.read()
    assert b[:8] == b"MRCQRSEL"
    off = 16 + 2 * 4 * SO.NUM_FEATURES
    return [float(x) for x in np.frombuffer(b[off:off + 12], "<f4")]


def test_shipped_selector_saves_work_on_held_out_mix(env):
    """AUTO with the shipped weights on matrices outside the training set:
    every factorization succeeds (escalation covers a low choice), and the
    ladder cost of the chosen starts, at the run costs stored with the
    weights, is well below always starting at FP32 and at most that of
    always starting at FP64."""
    torch, M, S = env
    S.load_into_library()
    costs = _shipped_costs(S)
    assert costs[0] == 1.0 and costs[0] <= costs[1] <= costs[2]
    rng = np.random.default_rng(77)
    m = 1 << 14
    tot = {"auto": 0.0, "fp32": 0.0, "fp64": 0.0}
    levels = ["fp16", "fp32", "fp64"]
    for i in range(48):
        n = int(rng.choice([48, 96, 160]))
        kind = inputs.SPECTRA[int(rng.integers(len(inputs.SPECTRA)))]
        kappa = float(10.0 ** rng.uniform(0.0, 16.0))
        A = inputs.make_matrix_torch(m, n, kappa, kind=kind, seed=7_000_003 + i, device="cuda")
        Q = M.empty_colmajor(m, n)
        R = M.empty_colmajor(n, n)
        M.factor_ex(A, Q, R, prec="auto", seed=i)
        st = M.last_status()
        assert st["status"] == "OK", (i, n, kappa, kind, st)
        first, used = levels.index(st["prec_first"]), levels.index(st["prec_used"])
        tot["auto"] += sum(costs[first:used + 1])
        label = 0 if S.passes(A, "fp16", seed=i) else (1 if S.passes(A, "fp32", seed=i) else 2)
        tot["fp32"] += costs[1] if label <= 1 else costs[1] + costs[2]
        tot["fp64"] += costs[2]
    assert tot["auto"] <= 0.9 * tot["fp32"], tot
    assert tot["auto"] <= tot["fp64"], tot


def test_selector_gain_in_measured_time(env):
    """What the trained network gains, in measured wall time with its own
    FP16 sketch and features included: 48 held-out matrices at m = 2^20
    (n in {64, 128, 256}, kappa_2 log-uniform in [1, 1e16]) factored under
    AUTO and under the fixed starts of the precision ladder without it.
    AUTO avoids the failed low-precision runs of always-FP16 and
    always-FP32, and costs no more than always-FP64 (the FP64 sketch is
    only 1.2-1.5 FP16 runs with emulated FP64 products, so that margin is
    small)."""
    torch, M, S = env
    r = S.policy_times(48, 1 << 20, seed0=5, reps=1)
    assert all(r["all_ok"].values()), r
    t = r["total_ms"]
    assert t["auto"] <= 0.75 * t["fp16"], r
    assert t["auto"] <= 0.9 * t["fp32"], r
    assert t["auto"] <= 1.05 * t["fp64"], r
