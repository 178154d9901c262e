"""Regime estimates without learning (Sec. II-C) through the C ABI, against
the oracle: the CholQR probe bound and the block 1-norm estimate on A^T A.

The 1-norm estimate follows the same steps with the same Philox columns on
both sides, so the estimates agree to the rounding of the substitutions
(relative error about kappa(A^T A) u); ||A^T A||_1 agrees to rounding.  The
probe's q measures CholQR's own loss of orthogonality, which differs between
two implementations by a modest factor, so its kappa is compared within a
factor; the regimes agree wherever the estimate is not near a threshold."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_18411_gb300 import build
    build.build()
    from paper_2606_18411_gb300 import mrcqr
    return mrcqr


def _est(M, A, method, seed=0):
    out = M.regime_estimate(M.to_colmajor(A), method, seed=seed)
    return out.cpu().numpy()


def _near_threshold(kappa):
    return any(abs(math.log10(kappa) - t) < 0.3 for t in (4.0, 8.0))


@pytest.mark.parametrize("kappa", [1e0, 1e3, 1e6])
@pytest.mark.parametrize("m,n", [(4096, 24), (10007, 100), (20000, 257)])
def test_onenorm_against_oracle(M, m, n, kappa):
    A = inputs.make_matrix(m, n, kappa, seed=n)
    got = _est(M, A, "onenorm", seed=7)
    ref_kappa, ref_g1, ref_est = O.onenorm_regime_estimate(A, seed=7)
    assert got[2] == pytest.approx(ref_g1, rel=1e-12)
    kG = kappa ** 2
    assert got[3] == pytest.approx(ref_est, rel=max(1e-10, 1e3 * kG * O.U_FP64))
    assert got[0] == pytest.approx(ref_kappa, rel=max(1e-10, 1e3 * kG * O.U_FP64))
    G = A.T @ A
    exact = np.abs(np.linalg.inv(G)).sum(axis=0).max()   # itself accurate to about kappa(G) u
    assert got[3] <= exact * (1 + 1e-10 + 1e3 * kG * O.U_FP64)   # the estimator's lower-bound property
    if not _near_threshold(ref_kappa):
        assert int(got[1]) == O.regime_of(ref_kappa)


@pytest.mark.parametrize("n", [1, 3, 4])
def test_onenorm_exact_for_tiny_n(M, n):
    A = inputs.make_matrix(1000, n, 1e3, seed=n)
    got = _est(M, A, "onenorm")
    exact = np.abs(np.linalg.inv(A.T @ A)).sum(axis=0).max()
    assert got[3] == pytest.approx(exact, rel=1e-8)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("m,n", [(4096, 32), (20000, 120)])
def test_probe_against_oracle(M, m, n, kappa):
    A = inputs.make_matrix(m, n, kappa, seed=n + 1)
    got = _est(M, A, "probe")
    ref_kappa, ref_q = O.cholqr_probe(A)
    # q is CholQR's own loss of orthogonality: the device's once-rounded Gram moves it by a factor
    # of about 2 against numpy's, and the power iteration approaches q from below
    assert ref_kappa / 5 <= got[0] <= 5 * ref_kappa, (got, ref_kappa)
    assert got[0] <= 2 * O.cond2(A)     # a lower bound up to the constant of CholQR's error bound
    if not _near_threshold(ref_kappa):
        assert int(got[1]) == O.regime_of(ref_kappa)


@pytest.mark.parametrize("method", ["probe", "onenorm"])
def test_breakdown_means_double(M, method):
    # kappa_2 = 1e12: the Gram matrix (kappa 1e24) is numerically singular; the Cholesky factorization
    # breaks down (kappa = inf) or ends on rounding noise with a huge estimate
    A = inputs.make_matrix(8192, 40, 1e12, seed=2)
    got = _est(M, A, method)
    assert got[1] == 2.0 and (math.isinf(got[0]) or got[0] > 1e8), got


def test_invalid_arguments(M):
    import torch
    from paper_2606_18411_gb300 import _lib
    lib = _lib.load()
    A = M.to_colmajor(inputs.gaussian(64, 8, seed=0))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    assert lib.mrcqr_regime_estimate(64, 8, A.data_ptr(), 64, 2, 0, out.data_ptr(), None) == 1   # no such method
    assert lib.mrcqr_regime_estimate(4, 8, A.data_ptr(), 64, 0, 0, out.data_ptr(), None) == 1    # m < n
    assert lib.mrcqr_regime_estimate(64, 8, A.data_ptr(), 63, 1, 0, out.data_ptr(), None) == 1   # lda < m
