"""Parity at the full sizes of the large-factorization workloads, through the
C ABI and in the launch configuration the bench times (mrcqr_factor_ex with
the device judge and escalation on, s = 2n, inputs from the bench's device
generator).

* m = 2^20, n in {64, 128, 256, 512}, geometric spectra with kappa_2 in
  {1e2, 1e4, 1e8, 1e12, 1e16}, sketch precision by the paper's bounds
  (FP16 up to 1e4, FP32 up to 1e8, FP64 above; Sec. II-B).
* m = 2^22, n = 128, geometric / step-cliff / clustered spectra, every sketch
  precision (FP16, BF16, FP32, FP64), with and without escalation.

The oracle cannot factor these in seconds, so it checks sampled outputs it
can compute one by one, each in double-double (Dot2):
* the Gram matrix of a sample of Q's columns (a principal submatrix of
  Q^T Q, so its distance from I is at most ||I - Q^T Q||_2);
* the residual of the leading column block: R is upper triangular, so
  A[:, :k] = Q[:, :k] R[:k, :k] exactly;
* sampled entries of the sketch Y = sqrt(m/s) P F D A against the oracle's
  dense sketch rows (Algorithm 2 steps 1-4)."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13
SKETCH_TOL = {"fp16": 5e-3, "bf16": 5e-3, "fp32": 1e-5, "fp64": 1e-13}
SAFE = {"fp16": 1e4, "bf16": 1e2, "fp32": 1e8, "fp64": 1e16}   # largest kappa each precision is run at by rule


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_18411_gb300 import build
    build.build()
    from paper_2606_18411_gb300 import mrcqr
    return torch, mrcqr


def _factor(torch, M, A, prec, seed=0, escalate=True):
    m, n = A.shape
    Q = M.empty_colmajor(m, n, device=A.device)
    R = M.empty_colmajor(n, n, device=A.device)
    stats = torch.zeros(8, dtype=torch.float64, device=A.device)
    M.factor_ex(A, Q, R, prec=prec, seed=seed, escalate=escalate, stats_device=stats)
    torch.cuda.synchronize()
    from paper_2606_18411_gb300 import _lib
    st = _lib.Stats.from_buffer_copy(stats.cpu().numpy().tobytes()).as_dict()
    return Q, R, st


def _sampled_checks(A, Q, R, k_lead, n_extra, seed):
    """(orthogonality of sampled columns (2-norm), residual of the leading block (Frobenius))."""
    n = A.shape[1]
    rng = np.random.default_rng(seed)
    k = min(n, k_lead)
    cols = np.unique(np.concatenate([np.arange(k), rng.choice(n, min(n, n_extra), replace=False)]))
    o2, _, _ = O.orthogonality_error(Q[:, cols.tolist()].cpu().numpy())
    rf, _ = O.residual_error(A[:, :k].cpu().numpy(), Q[:, :k].cpu().numpy(), R[:k, :k].cpu().numpy())
    return o2, rf


def _r_is_upper_positive(R):
    Rh = R.cpu().numpy()
    return bool(np.all(np.tril(Rh, -1) == 0) and np.all(np.diag(Rh) > 0))


@pytest.mark.parametrize("n", [64, 128, 256, 512])
def test_large_factorizations_rule_precision(env, n):
    torch, M = env
    m = 1 << 20
    for i, kappa in enumerate([1e2, 1e4, 1e8, 1e12, 1e16]):
        prec = O.precision_rule(kappa)
        A = inputs.make_matrix_device(m, n, kappa, seed=2000 + 10 * n + i, device="cuda")
        Q, R, st = _factor(torch, M, A, prec)
        assert st["status"] == "OK" and st["ortho_fro"] <= TOL, (n, kappa, st)
        if kappa < SAFE[prec]:
            assert st["retries"] == 0 and st["prec_used"] == prec, (n, kappa, st)
        else:
            # at the regime boundary (FP16 at 1e4, FP32 at 1e8: u_p kappa ~ 5) the sketch may miss the
            # bound by a little; the judge then re-sketches once at the next precision (Sec. II-C)
            assert st["retries"] <= 1, (n, kappa, st)
        o2, rf = _sampled_checks(A, Q, R, k_lead=32, n_extra=16, seed=n + i)
        assert o2 <= TOL and rf <= TOL, (n, kappa, o2, rf)
        assert _r_is_upper_positive(R)
        if kappa <= 1e8:
            # R[:16, :16] is the R factor of A[:, :16] (R upper triangular): against the
            # oracle's Householder QR of those columns, O(kappa u) apart
            Rl = R[:16, :16].cpu().numpy()
            Rref = O.householder_qr(A[:, :16].cpu().numpy())
            err = float(np.linalg.norm(Rl - Rref) / np.linalg.norm(Rref))
            assert err <= 100 * kappa * O.U_FP64, (n, kappa, err)
        del A, Q, R
        torch.cuda.empty_cache()


def _oracle_sketch_entries(A, idx, signs, rows, cols):
    """Y[rows, cols] of the FP64 oracle sketch, from dense rows of S."""
    m = A.shape[0]
    s = len(idx)
    Ac = A[:, cols.tolist()].cpu().numpy()
    return np.stack([O.sketch_row(int(idx[r]), m, s, signs) @ Ac for r in rows])


@pytest.mark.parametrize("kind", ["geometric", "cliff", "clustered"])
def test_precision_sweep_m4194304(env, kind):
    torch, M = env
    m, n, s, seed = 1 << 22, 128, 256, 0
    idx = O.sample_rows(m, s, seed)
    signs = O.rademacher(m, seed)
    rng = np.random.default_rng(7)
    rows = rng.choice(s, 6, replace=False)
    cols = rng.choice(n, 6, replace=False)
    for kappa in [1e0, 1e4, 1e8, 1e12, 1e16]:
        A = inputs.make_matrix_device(m, n, kappa, kind=kind, seed=3000 + int(round(math.log10(kappa))), device="cuda")
        Yref = _oracle_sketch_entries(A, idx, signs, rows, cols)
        for prec in ["fp16", "bf16", "fp32", "fp64"]:
            # the sketch against the FP64 oracle (sampled entries, relative to their norm)
            Y = M.sketch(A, s, prec=prec, seed=seed).cpu().numpy()[np.ix_(rows, cols)]
            err = float(np.linalg.norm(Y - Yref) / np.linalg.norm(Yref))
            assert err <= SKETCH_TOL[prec], (kind, kappa, prec, err)
            # with escalation the result meets the bound from every starting precision (Sec. II-C)
            Q, R, st = _factor(torch, M, A, prec, seed=seed)
            assert st["status"] == "OK" and st["ortho_fro"] <= TOL, (kind, kappa, prec, st)
            o2, rf = _sampled_checks(A, Q, R, k_lead=16, n_extra=8, seed=int(kappa % 97))
            assert o2 <= TOL and rf <= TOL, (kind, kappa, prec, o2, rf)
            if kappa * 1e2 <= SAFE[prec]:   # well inside the precision's regime: no re-sketch
                assert st["retries"] == 0, (kind, kappa, prec, st)
            del Q, R
            # without escalation: far outside a precision's regime it cannot reach the bound
            if prec != "fp64" and kappa >= 1e8 * SAFE[prec]:
                Q, R, st = _factor(torch, M, A, prec, seed=seed, escalate=False)
                assert st["status"] != "OK", (kind, kappa, prec, st)
                del Q, R
        del A
        torch.cuda.empty_cache()
