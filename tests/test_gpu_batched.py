"""Batched MRCQR (grouped launches over many problems of uneven m and n)
against the CPU oracle's checks and the single-matrix entry point."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
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
    return torch, M


def _batch(shapes, seed0=500):
    mats, kappas = [], []
    for i, (m, n, kappa) in enumerate(shapes):
        mats.append(inputs.make_matrix(m, n, kappa, seed=seed0 + i))
        kappas.append(kappa)
    return mats, kappas


SHAPES = [(16384, 16, 1e0), (20001, 32, 1e3), (16384, 64, 1e6), (30000, 128, 1e9), (5000, 50, 1e11),
          (16384, 16, 1e12), (40000, 100, 1e2), (12288, 128, 1e4), (9999, 7, 1e7), (16384, 33, 1e10)]


def _run_oneshot(torch, M, mats, precs, seeds):
    As = [M.to_colmajor(a) for a in mats]
    Qs = [M.empty_colmajor(*a.shape) for a in mats]
    Rs = [M.empty_colmajor(a.shape[1], a.shape[1]) for a in mats]
    status = torch.full((len(mats),), -1, dtype=torch.int32, device="cuda")
    M.factor_batched(As, Qs, Rs, precs, seeds, status)
    torch.cuda.synchronize()
    return As, Qs, Rs, status


def test_batched_rule_precision_against_oracle(env):
    torch, M = env
    mats, kappas = _batch(SHAPES)
    precs = [O.precision_rule(k) for k in kappas]
    _, Qs, Rs, status = _run_oneshot(torch, M, mats, precs, list(range(len(mats))))
    assert status.cpu().tolist() == [0] * len(mats)
    for A, Q, R, k in zip(mats, Qs, Rs, kappas):
        Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
        assert O.orthogonality_error(Qh)[0] <= 1e-13, k
        assert O.residual_error(A, Qh, Rh)[0] <= 1e-13, k
        assert np.all(np.diag(Rh) > 0)


def test_batched_matches_single_factorizations(env):
    torch, M = env
    mats, kappas = _batch(SHAPES[:6], seed0=900)
    precs = [O.precision_rule(k) for k in kappas]
    _, Qs, Rs, status = _run_oneshot(torch, M, mats, precs, [7] * len(mats))
    for A, Qb, Rb, p in zip(mats, Qs, Rs, precs):
        Q1, R1 = M.factor(M.to_colmajor(A), prec=p, seed=7)
        # same sign vector and sample set; only summation orders differ
        assert np.linalg.norm(Rb.cpu().numpy() - R1.cpu().numpy()) <= 1e-9 * np.linalg.norm(R1.cpu().numpy())


def test_batched_escalates_per_problem(env):
    torch, M = env
    mats, kappas = _batch([(16384, 32, 1e2), (16384, 32, 1e13), (20000, 64, 1e3)], seed0=1300)
    # the middle problem is given a precision far too low and must escalate alone
    _, Qs, Rs, status = _run_oneshot(torch, M, mats, ["fp16", "fp16", "bf16"], [1, 2, 3])
    assert status.cpu().tolist() == [0, 0, 0]
    for A, Q, R in zip(mats, Qs, Rs):
        assert O.orthogonality_error(Q.cpu().numpy())[0] <= 1e-13
        assert O.residual_error(A, Q.cpu().numpy(), R.cpu().numpy())[0] <= 1e-13


def test_batched_plan_graph_replay_and_autotune(env):
    torch, M = env
    mats, kappas = _batch(SHAPES[:5], seed0=1700)
    precs = [O.precision_rule(k) for k in kappas]
    As = [M.to_colmajor(a) for a in mats]
    Qs = [M.empty_colmajor(*a.shape) for a in mats]
    Rs = [M.empty_colmajor(a.shape[1], a.shape[1]) for a in mats]
    status = torch.full((len(mats),), -1, dtype=torch.int32, device="cuda")
    plan = M.BatchedPlan(As, Qs, Rs, precs, [3] * len(mats), status, use_graph=True, autotune=True)
    info = plan.info()
    assert info["rows_per_split"] in (1024, 2048, 4096, 8192)
    assert info["rows_per_chunk"] in (2048, 4096, 8192, 16384)
    for rep in range(2):
        if rep == 1:
            # new data in the same buffers: the captured graph reads them
            mats = [inputs.make_matrix(a.shape[0], a.shape[1], k, seed=2500 + i)
                    for i, (a, k) in enumerate(zip(mats, kappas))]
            for Ad, a in zip(As, mats):
                Ad.copy_(torch.from_numpy(a))
        status.fill_(-1)
        plan.execute()
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0] * len(mats)
        for A, Q, R in zip(mats, Qs, Rs):
            assert O.orthogonality_error(Q.cpu().numpy())[0] <= 1e-13
            assert O.residual_error(A, Q.cpu().numpy(), R.cpu().numpy())[0] <= 1e-13
    plan.close()


def test_batched_plan_grouped_fp64_fma_mode(env):
    # fp64_products = 1: every phase grouped with FP64 FMA kernels; same bounds, same statuses
    torch, M = env
    mats, kappas = _batch(SHAPES[:5], seed0=1900)
    precs = [O.precision_rule(k) for k in kappas]
    As = [M.to_colmajor(a) for a in mats]
    Qs = [M.empty_colmajor(*a.shape) for a in mats]
    Rs = [M.empty_colmajor(a.shape[1], a.shape[1]) for a in mats]
    status = torch.full((len(mats),), -1, dtype=torch.int32, device="cuda")
    plan = M.BatchedPlan(As, Qs, Rs, precs, [5] * len(mats), status, use_graph=True, fp64_products=1)
    plan.execute()
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(mats)
    for A, Q, R in zip(mats, Qs, Rs):
        assert O.orthogonality_error(Q.cpu().numpy())[0] <= 1e-13
        assert O.residual_error(A, Q.cpu().numpy(), R.cpu().numpy())[0] <= 1e-13
    plan.close()


def test_batched_rejects_invalid(env):
    torch, M = env
    A = M.to_colmajor(inputs.gaussian(100, 60, seed=1))   # m < 2n
    Q = M.empty_colmajor(100, 60)
    R = M.empty_colmajor(60, 60)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MrcqrError):
        M.factor_batched([A], [Q], [R], ["fp64"], [0], status)


@pytest.mark.parametrize("fp64_products", [0, 1])
@pytest.mark.parametrize("transform", ["rfft", "rfft_reim"])
def test_batched_plan_paper_transform(env, transform, fp64_products):
    # the paper's real-FFT sketch (2n bins per problem) in a batched plan
    torch, M = env
    mats, kappas = _batch(SHAPES[:6], seed0=2100)
    precs = [O.precision_rule(k) for k in kappas]
    As = [M.to_colmajor(a) for a in mats]
    Qs = [M.empty_colmajor(*a.shape) for a in mats]
    Rs = [M.empty_colmajor(a.shape[1], a.shape[1]) for a in mats]
    status = torch.full((len(mats),), -1, dtype=torch.int32, device="cuda")
    plan = M.BatchedPlan(As, Qs, Rs, precs, [3] * len(mats), status, use_graph=True, fp64_products=fp64_products,
                         transform=transform)
    plan.execute()
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(mats)
    for A, Q, R, p in zip(mats, Qs, Rs, precs):
        Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
        assert O.orthogonality_error(Qh)[0] <= 1e-13
        assert O.residual_error(A, Qh, Rh)[0] <= 1e-13
        if fp64_products == 0:
            # the same bins, signs and kernels as a single call with that transform: summation order only
            _, R1 = M.factor(M.to_colmajor(A), prec=p, seed=3, transform=transform, s_factor=2)
            R1h = R1.cpu().numpy()
            assert np.linalg.norm(Rh - R1h) <= 1e-9 * np.linalg.norm(R1h)
    plan.close()


def test_batched_plan_rejects_too_few_bins(env):
    # 2n = 60 bins of a real column with m = 100 (51 distinct bins) do not exist; the DCT plan is fine
    torch, M = env
    A = M.to_colmajor(inputs.gaussian(100, 30, seed=2))
    Q = M.empty_colmajor(100, 30)
    R = M.empty_colmajor(30, 30)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MrcqrError):
        M.BatchedPlan([A], [Q], [R], ["fp64"], [0], status, transform="rfft")
    plan = M.BatchedPlan([A], [Q], [R], ["fp64"], [0], status)
    plan.execute()
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0]
    plan.close()


def test_grouped_heavy_phases_match_per_problem_kernels(env):
    # the emulated-FP64 heavy phases as grouped persistent launches (the default) against the same
    # single-problem kernels run per problem on side streams: the per-item arithmetic is the same and
    # the Gram and check sums are exact integer sums, so Q and R agree bit for bit; the grouped plan
    # launches a fixed number of kernels per phase instead of several per problem
    torch, M = env
    shapes = SHAPES + [(70000, 200, 1e13), (33333, 96, 1e5)]
    mats, kappas = _batch(shapes, seed0=2100)
    precs = [O.precision_rule(k) for k in kappas]
    precs[3] = "fp16"   # kappa 1e9 from FP16: escalates inside the grouped launches
    As = [M.to_colmajor(a) for a in mats]
    out = {}
    for per_problem in (0, 1):
        Qs = [M.empty_colmajor(*a.shape) for a in mats]
        Rs = [M.empty_colmajor(a.shape[1], a.shape[1]) for a in mats]
        status = torch.full((len(mats),), -1, dtype=torch.int32, device="cuda")
        plan = M.BatchedPlan(As, Qs, Rs, precs, list(range(len(mats))), status, use_graph=True,
                             oz_per_problem=per_problem)
        plan.execute()
        torch.cuda.synchronize()
        assert status.cpu().tolist() == [0] * len(mats), per_problem
        out[per_problem] = ([q.cpu().numpy() for q in Qs], [r.cpu().numpy() for r in Rs], plan.info())
        plan.close()
    for qg, qp, rg, rp in zip(out[0][0], out[1][0], out[0][1], out[1][1]):
        np.testing.assert_array_equal(qg, qp)
        np.testing.assert_array_equal(rg, rp)
    for A, Q, R in zip(mats, out[0][0], out[0][1]):
        assert O.orthogonality_error(Q)[0] <= 1e-13
        assert O.residual_error(A, Q, R)[0] <= 1e-13
    assert out[0][2]["kernels_per_execute"] < 120 < out[1][2]["kernels_per_execute"], (out[0][2], out[1][2])


@pytest.mark.parametrize("rows_per_chunk", [2048, 8192])
def test_batched_mixes_tma_and_plain_copy_sketches(env, rows_per_chunk):
    # even m (TMA loads of A) and odd m (plain copies: no TMA map for an odd leading dimension) share the
    # grouped tensor-core sketch launches, so a CTA runs items of both kinds in turn; with escalation off
    # every FP16 / BF16 / FP32 sketch must be right the first time, and Q, R pass the oracle's checks
    torch, M = env
    shapes = [(16384, 32, 1e2, "fp16"), (16385, 32, 1e2, "fp16"), (20001, 48, 1e3, "fp16"), (20000, 48, 1e3, "fp16"),
              (12289, 100, 1e2, "fp16"), (12288, 100, 1e2, "fp16"), (9999, 16, 1e1, "bf16"), (10000, 16, 1e1, "bf16"),
              (30001, 64, 1e5, "fp32"), (30000, 64, 1e5, "fp32"), (8191, 130, 1e4, "fp32"), (8192, 130, 1e4, "fp32")]
    mats = [inputs.make_matrix(m, n, k, seed=2100 + i) for i, (m, n, k, _) in enumerate(shapes)]
    precs = [p for *_, p in shapes]
    As = [M.to_colmajor(a) for a in mats]
    Qs = [M.empty_colmajor(*a.shape) for a in mats]
    Rs = [M.empty_colmajor(a.shape[1], a.shape[1]) for a in mats]
    status = torch.full((len(mats),), -1, dtype=torch.int32, device="cuda")
    plan = M.BatchedPlan(As, Qs, Rs, precs, list(range(len(mats))), status, escalate=False,
                         rows_per_chunk=rows_per_chunk)
    for _ in range(2):
        plan.execute()
    torch.cuda.synchronize()
    plan.close()
    assert status.cpu().tolist() == [0] * len(mats)
    for A, Q, R in zip(mats, Qs, Rs):
        Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
        assert O.orthogonality_error(Qh)[0] <= 1e-13
        assert O.residual_error(A, Qh, Rh)[0] <= 1e-13


def test_batched_512_problem_distribution_against_oracle(env):
    # the batched workload's own distribution: 512 problems, m uniform in [2^14, 2^18], n in
    # {16, 32, 64, 128}, geometric spectra with kappa log-uniform in [1, 1e12], precision by rule, one
    # grouped plan replayed as a CUDA graph; every problem must report OK with diag(R) > 0, and 16 of
    # them (the largest and smallest m, the rest drawn) pass the oracle's double-double orthogonality
    # and residual checks
    torch, M = env
    rng = np.random.default_rng(4000)
    cnt = 512
    ms = rng.integers(1 << 14, (1 << 18) + 1, cnt)
    ns = rng.choice([16, 32, 64, 128], cnt)
    kap = 10.0 ** rng.uniform(0.0, 12.0, cnt)
    As = [inputs.make_matrix_torch(int(mm), int(nn), float(k), seed=7000 + i, device="cuda")
          for i, (mm, nn, k) in enumerate(zip(ms, ns, kap))]
    Qs = [M.empty_colmajor(int(mm), int(nn)) for mm, nn in zip(ms, ns)]
    Rs = [M.empty_colmajor(int(nn), int(nn)) for nn in ns]
    status = torch.full((cnt,), -1, dtype=torch.int32, device="cuda")
    precs = [O.precision_rule(float(k)) for k in kap]
    plan = M.BatchedPlan(As, Qs, Rs, precs, list(range(cnt)), status, use_graph=True)
    plan.execute()
    torch.cuda.synchronize()
    plan.close()
    assert status.cpu().tolist() == [0] * cnt
    for R in Rs:
        assert bool(torch.all(torch.diagonal(R) > 0))
    pick = {int(np.argmax(ms)), int(np.argmin(ms))}
    pick |= set(int(i) for i in rng.choice(cnt, 14, replace=False))
    for i in sorted(pick):
        A, Q, R = As[i].cpu().numpy(), Qs[i].cpu().numpy(), Rs[i].cpu().numpy()
        assert O.orthogonality_error(Q)[0] <= 1e-13, (i, ms[i], ns[i], kap[i])
        assert O.residual_error(A, Q, R)[0] <= 1e-13, (i, ms[i], ns[i], kap[i])
