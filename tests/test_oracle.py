"""Pins of the CPU oracle against what the paper and the mathematics fix
(no GPU).  Each test names the passage it follows."""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import oracle as O
from paper_2606_18411_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- Algorithm 2 step 1: random signs and sample set (Philox, Floyd) ---------

def test_philox_known_answers():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0], v[1], v[2], v[3], v[4], v[5])
        assert [int(x) for x in out] == v[6:10]


def test_philox_vectorised_matches_scalar():
    ctr = np.arange(1000, 1016, dtype=np.uint64)
    vec = O.philox4x32_10(ctr, 7, 0, 3, 0x12345678, 0x9abcdef0)
    for i, c in enumerate(ctr.tolist()):
        sc = O.philox4x32_10(c, 7, 0, 3, 0x12345678, 0x9abcdef0)
        assert [int(x[i]) for x in vec] == [int(x) for x in sc]


@pytest.mark.parametrize("m", [1, 7, 4096, 1 << 16])
def test_rademacher_signs(m):
    d = O.rademacher(m, seed=11)
    assert d.shape == (m,)
    assert set(np.unique(d).tolist()) <= {-1.0, 1.0}
    assert abs(d.sum()) <= 5 * math.sqrt(m) + 1
    # different seeds give different sign vectors
    if m >= 64:
        assert not np.array_equal(d, O.rademacher(m, seed=12))


@pytest.mark.parametrize("m,s", [(1, 1), (5, 5), (64, 64), (4096, 64), (1 << 20, 256), (3001, 2048)])
def test_sample_rows_valid(m, s):
    idx = O.sample_rows(m, s, seed=3)
    assert idx.shape == (s,)
    assert np.all(np.diff(idx) > 0)          # sorted, distinct
    assert idx[0] >= 0 and idx[-1] < m
    if s == m:
        assert np.array_equal(idx, np.arange(m))


def test_sample_rows_uniform_subsets():
    # Floyd's algorithm draws every s-subset with probability 1/C(m,s).
    m, s, trials = 5, 2, 6000
    counts = {}
    for seed in range(trials):
        key = tuple(O.sample_rows(m, s, seed).tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == math.comb(m, s)
    exp = trials / math.comb(m, s)
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 30.0          # 9 dof; p ~ 4e-4


def test_sample_rows_deterministic():
    assert np.array_equal(O.sample_rows(10000, 100, 5), O.sample_rows(10000, 100, 5))
    assert not np.array_equal(O.sample_rows(10000, 100, 5), O.sample_rows(10000, 100, 6))


# --- Algorithm 2 steps 2-4: the orthonormal DCT-II sketch ---------------------

@pytest.mark.parametrize("m", [8, 64, 256, 300])
def test_dct_matches_library_and_is_orthonormal(m):
    F = O.dct_matrix(m)
    np.testing.assert_allclose(F @ F.T, np.eye(m), atol=1e-13)
    x = inputs.gaussian(m, 3, seed=m)
    ref = scipy.fft.dct(x, type=2, norm="ortho", axis=0)
    np.testing.assert_allclose(F @ x, ref, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("m,n", [(256, 8), (300, 5), (1024, 16)])
def test_sketch_equals_fast_transform(m, n):
    # Y = sqrt(m/s) P F D A, computed independently with scipy's DCT
    s = 2 * n
    A = inputs.gaussian(m, n, seed=1)
    d = O.rademacher(m, 9)
    idx = O.sample_rows(m, s, 9)
    Y = O.sketch(A, idx, d)
    ref = math.sqrt(m / s) * scipy.fft.dct(d[:, None] * A, type=2, norm="ortho", axis=0)[idx]
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_sketch_full_sample_preserves_gram():
    # with s = m and every row sampled, S^T S = (m/s) I = I: Y^T Y = A^T A
    m, n = 128, 6
    A = inputs.gaussian(m, n, seed=2)
    Y = O.sketch(A, O.sample_rows(m, m, 1), O.rademacher(m, 1))
    np.testing.assert_allclose(Y.T @ Y, A.T @ A, atol=1e-12)


# --- The paper's real-FFT sketch (Algorithm 2 as printed, Sec. II-A) ----------

@pytest.mark.parametrize("m", [1, 2, 7, 64, 1000, 1025])
def test_rfft_rows_match_library(m):
    # Re and Im of every row of the unnormalised DFT against numpy's real FFT
    x = inputs.gaussian(m, 3, seed=m)
    ref = np.fft.rfft(x, axis=0)
    assert ref.shape[0] == m // 2 + 1
    Re = np.stack([O.rfft_re_row(k, m) for k in range(m // 2 + 1)])
    Im = np.stack([O.rfft_im_row(k, m) for k in range(m // 2 + 1)])
    tol = 1e-13 * np.abs(x).sum(axis=0).max()
    np.testing.assert_allclose(Re @ x, ref.real, rtol=0, atol=tol)
    np.testing.assert_allclose(Im @ x, ref.imag, rtol=0, atol=tol)


@pytest.mark.parametrize("m,c", [(1, 1), (2, 2), (7, 4), (64, 33), (4096, 150), (1 << 17, 150), (3001, 1501)])
def test_sample_bins_valid(m, c):
    # c distinct bins of the floor(m/2) + 1 that a real column has (Hermitian symmetry)
    b = O.sample_bins(m, c, seed=5)
    assert b.shape == (c,)
    assert np.all(np.diff(b) > 0) and b[0] >= 0 and b[-1] <= m // 2
    if c == m // 2 + 1:
        assert np.array_equal(b, np.arange(m // 2 + 1))


def test_sample_bins_uniform_subsets():
    # m = 8 has 5 distinct bins; each 2-subset of them is drawn with probability 1/10
    m, c, trials = 8, 2, 5000
    counts = {}
    for seed in range(trials):
        key = tuple(O.sample_bins(m, c, seed).tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == math.comb(5, 2) and all(max(k) <= 4 for k in counts)
    exp = trials / math.comb(5, 2)
    chi2 = sum((v - exp) ** 2 / exp for v in counts.values())
    assert chi2 < 30.0          # 9 dof; p ~ 4e-4


@pytest.mark.parametrize("m,n", [(256, 8), (301, 5), (1024, 16)])
def test_rfft_sketch_equals_fast_transform(m, n):
    # Y = sqrt(c/m) Re(FFT(D A))[bins] (and the Im rows below), independently with numpy's real FFT
    c = 3 * n
    A = inputs.gaussian(m, n, seed=1)
    d = O.rademacher(m, 9)
    bins = O.sample_bins(m, c, 9)
    F = np.fft.rfft(d[:, None] * A, axis=0)[bins]
    ref = math.sqrt(c / m) * np.concatenate([F.real, F.imag])
    tol = 1e-13 * np.abs(ref).max()
    np.testing.assert_allclose(O.rfft_sketch(A, bins, d, imag=True), ref, rtol=0, atol=tol)
    np.testing.assert_allclose(O.rfft_sketch(A, bins, d), ref[:c], rtol=0, atol=tol)


@pytest.mark.parametrize("m", [64, 65])
def test_rfft_all_bins_parseval(m):
    # Parseval for real columns a, b with spectra X, Y: sum_k w_k (Re X_k Re Y_k + Im X_k Im Y_k) = m a^T b
    # over the floor(m/2) + 1 bins, w_k = 2 except w_0 = 1 and (m even) w_{m/2} = 1.  With every bin
    # sampled (c of them), the scale sqrt(c/m) and D^2 = I: Y^T W Y = c A^T A.
    n = 5
    c = m // 2 + 1
    A = inputs.gaussian(m, n, seed=3)
    d = O.rademacher(m, 4)
    bins = O.sample_bins(m, c, 4)
    Y = O.rfft_sketch(A, bins, d, imag=True)
    w = np.full(c, 2.0)
    w[0] = 1.0
    if m % 2 == 0:
        w[-1] = 1.0
    Wt = np.concatenate([w, w])
    G = c * (A.T @ A)
    np.testing.assert_allclose(Y.T @ (Wt[:, None] * Y), G, rtol=0, atol=1e-12 * np.abs(G).max())
    # the Im rows of bin 0 (and bin m/2 for even m) vanish
    assert np.all(Y[c] == 0)
    if m % 2 == 0:
        assert np.abs(Y[2 * c - 1]).max() <= 1e-12 * np.abs(Y).max()


@pytest.mark.parametrize("prec,tol", [("fp16", 5e-3), ("bf16", 5e-3), ("fp32", 1e-5)])
def test_emulated_rfft_sketch_within_precision_tolerance(prec, tol):
    m, n = 4096, 32
    A = inputs.make_matrix(m, n, 1e8, seed=4)
    d, bins = O.rademacher(m, 0), O.sample_bins(m, 3 * n, 0)
    Y = O.rfft_sketch(A, bins, d, imag=True)
    Yp = O.rfft_sketch_emulated(A, bins, d, prec, imag=True)
    err = np.linalg.norm(Yp - Y) / np.linalg.norm(Y)
    assert O.UNIT_ROUNDOFF[prec] / 100 < err < tol


# --- fl_p: rounding to the sketch precision (Algorithm 2 step 2) --------------

def test_round_significand_fp16_fp32_match_casts():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000) * np.exp2(rng.integers(-10, 12, 20000))
    x = x[(np.abs(x) >= 2.0 ** -14) & (np.abs(x) <= 65504.0)]   # FP16 normal range
    np.testing.assert_array_equal(O.round_significand(x, 11), x.astype(np.float16).astype(np.float64))
    y = rng.standard_normal(20000) * np.exp2(rng.integers(-100, 100, 20000))
    np.testing.assert_array_equal(O.round_significand(y, 24), y.astype(np.float32).astype(np.float64))


def test_round_significand_bf16_matches_torch_on_fp32_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * np.exp2(rng.integers(-30, 30, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.round_significand(x.astype(np.float64), 8), ref)


def test_round_significand_ties_to_even():
    one = 1.0
    ulp16 = 2.0 ** -10
    assert O.round_significand(np.array([one + ulp16 / 2]), 11)[0] == one
    assert O.round_significand(np.array([one + 1.5 * ulp16]), 11)[0] == one + 2 * ulp16
    assert O.round_significand(np.array([-(one + 1.5 * ulp16)]), 11)[0] == -(one + 2 * ulp16)


@pytest.mark.parametrize("prec,tol", [("fp16", 5e-3), ("bf16", 5e-3), ("fp32", 1e-5)])
def test_emulated_sketch_within_precision_tolerance(prec, tol):
    m, n = 4096, 32
    A = inputs.make_matrix(m, n, 1e8, seed=4)
    d, idx = O.rademacher(m, 0), O.sample_rows(m, 2 * n, 0)
    Y = O.sketch(A, idx, d)
    Yp = O.sketch_emulated(A, idx, d, prec)
    err = np.linalg.norm(Yp - Y) / np.linalg.norm(Y)
    assert err < tol
    assert err > O.UNIT_ROUNDOFF[prec] / 100     # really rounded


# Exact special cases of the precision-p sketch models: where every rounding they model is exact, they
# must give the FP64 sketch bit for bit.  Bins 0 and m/2 of the real FFT have entries 1 and (-1)^j; DCT
# row 0 is the constant 1/sqrt(m); small-integer entries survive fl_p after the column scale 2^e; with
# m = 128 and c = 2 bins the scale sqrt(c/m) is 1/8, with m = 64 and s = 1 the DCT scale sqrt(m/s) is 8,
# so every product and sum is exact in FP64.  A dropped sign, scale or column exponent fails here.
@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_emulated_sketches_exact_where_rounding_is_exact(prec):
    rng = np.random.default_rng(11)
    A = rng.integers(-8, 9, size=(128, 6)).astype(np.float64)
    A[:, 2] *= 2.0 ** 40   # column scales far from 1
    A[:, 3] *= 2.0 ** -30
    d = O.rademacher(128, 7)
    bins = np.array([0, 64])
    np.testing.assert_array_equal(O.rfft_sketch_emulated(A, bins, d, prec), O.rfft_sketch(A, bins, d))
    B = A[:64]
    d2 = O.rademacher(64, 3)
    np.testing.assert_array_equal(O.sketch_emulated(B, np.array([0]), d2, prec), O.sketch(B, np.array([0]), d2))
    # the same call without the signs D differs: the models apply them
    assert not np.array_equal(O.rfft_sketch_emulated(A, bins, d, prec), O.rfft_sketch(A, bins, np.ones(128)))


# With entries that do round, the real-FFT model on bins {0, m/2} equals the FP64 sketch of D A whose
# scaled entries were rounded once to p (round_significand, pinned above against numpy and torch
# casts): the model rounds D A 2^e, not A, and undoes the scale exactly.
@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_emulated_rfft_sketch_rounds_the_scaled_signed_entries(prec):
    rng = np.random.default_rng(12)
    m, n = 128, 5
    A = rng.integers(-8, 9, size=(m, n)).astype(np.float64) + rng.integers(-2 ** 19, 2 ** 19, size=(m, n)) * 2.0 ** -20
    d = O.rademacher(m, 9)
    bins = np.array([0, m // 2])
    e = O.column_scale_exponents(A)
    bits = {"fp16": 11, "bf16": 8, "fp32": 24}[prec]
    Xr = np.ldexp(O.round_significand(d[:, None] * np.ldexp(A, e[None, :]), bits), -e[None, :])
    Y = O.rfft_sketch_emulated(A, bins, d, prec)
    np.testing.assert_array_equal(Y, O.rfft_sketch(d[:, None] * Xr, bins, d))
    assert not np.array_equal(Y, O.rfft_sketch(A, bins, d)) or prec == "fp32"   # the rounding is visible


# --- SketchQR, Cholesky, substitution (Algorithm 1, Algorithm 2 steps 5-9) ----

@pytest.mark.parametrize("c,n", [(8, 8), (64, 32), (300, 50)])
def test_householder_matches_library_qr(c, n):
    Y = inputs.gaussian(c, n, seed=c + n)
    Q, R = O.householder_qr(Y, want_q=True)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(np.tril(R, -1), 0)
    np.testing.assert_allclose(Q @ R, Y, atol=1e-13 * np.abs(Y).max())
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-13)
    _, Rl = np.linalg.qr(Y)
    Rl = Rl * np.sign(np.diag(Rl))[:, None]
    np.testing.assert_allclose(R, Rl, atol=1e-12 * np.abs(Rl).max())


def test_householder_fp32_and_row_permutation():
    Y = inputs.gaussian(96, 32, seed=5)
    R = O.householder_qr(Y)
    R32 = O.householder_qr(Y.astype(np.float32), dtype=np.float32)
    assert np.linalg.norm(R32 - R) / np.linalg.norm(R) < 1e-5
    perm = np.random.default_rng(0).permutation(96)
    np.testing.assert_allclose(O.householder_qr(Y[perm]), R, atol=1e-12 * np.abs(R).max())


def test_trsm_matches_library_and_identity():
    A = inputs.gaussian(500, 24, seed=6)
    R = inputs.upper_with_positive_diag(24, 1e3, seed=6)
    W = O.trsm_right_upper(A, R)
    ref = scipy.linalg.solve_triangular(R, A.T, trans="T", lower=False).T
    np.testing.assert_allclose(W, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_array_equal(O.trsm_right_upper(A, np.eye(24)), A)


def test_cholesky_matches_library_and_breaks_down():
    X = inputs.gaussian(200, 30, seed=7)
    G = X.T @ X
    R = O.cholesky_upper(G)
    np.testing.assert_allclose(R, np.linalg.cholesky(G).T, rtol=1e-12, atol=1e-12)
    with pytest.raises(O.CholeskyBreakdown):
        O.cholesky_upper(np.array([[1.0, 2.0], [2.0, 1.0]]))
    with pytest.raises(O.CholeskyBreakdown):
        Z = X.copy()
        Z[:, 3] = Z[:, 5]
        O.cholesky_upper(Z.T @ Z)


def test_cholqr_instability_and_probe_bound():
    # Algorithm 1: orthogonality O(kappa^2 u) (Sec. I-A); breakdown near 1e8
    m, n = 4096, 16
    q1 = O.orthogonality_error(O.cholqr(inputs.make_matrix(m, n, 1.0, seed=1))[0])[0]
    assert q1 < 1e-14
    for kappa in (1e2, 1e4, 1e6, 1e7):
        Q, _ = O.cholqr(inputs.make_matrix(m, n, kappa, seed=2))
        q = O.orthogonality_error(Q)[0]
        assert q < 100 * kappa ** 2 * O.U_FP64
        # probe of Sec. II-C: kappa >= sqrt(q / (u (1 + q)))
        assert O.probe_kappa_lower(q) <= kappa * 1.0000001
    if True:
        with pytest.raises(O.CholeskyBreakdown):
            O.cholqr(inputs.make_matrix(m, n, 1e10, seed=3))


def test_cholqr2_orthogonal_below_1e8_and_breaks_down_beyond():
    # CholQR2 (Sec. I-A): the second pass restores O(u) orthogonality while kappa^2 u < 1,
    # and the first Gram matrix is not positive definite in FP64 past kappa ~ 1e8
    m, n = 4096, 16
    for kappa in (1e0, 1e3, 1e6, 1e7):
        A = inputs.make_matrix(m, n, kappa, seed=5)
        Q, R = O.cholqr2(A)
        o2 = O.orthogonality_error(Q)[0]
        rf = O.residual_error(A, Q, R)[0]
        assert o2 < 1e-14 and rf < 1e-15, (kappa, o2, rf)
        # the unique thin QR with diag(R) > 0: LAPACK's Householder R, rows sign-normalised
        Rh = np.linalg.qr(A, mode="r")
        Rh = Rh * np.sign(np.diag(Rh))[:, None]
        assert np.linalg.norm(R - Rh) / np.linalg.norm(Rh) < 100 * kappa * O.U_FP64
    with pytest.raises(O.CholeskyBreakdown):
        O.cholqr2(inputs.make_matrix(m, n, 1e10, seed=6))


# --- Algorithm 2 end to end ---------------------------------------------------

@pytest.mark.parametrize("kappa", [1e0, 1e4, 1e8, 1e12, 1e16])
def test_mrcqr_fp64_sketch_orthogonal_and_backward_stable(kappa):
    m, n = 4096, 32
    A, U, sig, V = inputs.make_matrix(m, n, kappa, seed=10, return_factors=True)
    res = O.mrcqr(A, seed=0, prec="fp64")
    o2, of, _ = O.orthogonality_error(res.Q)
    rf, r2 = O.residual_error(A, res.Q, res.R)
    assert o2 <= 1e-13 and rf <= 1e-13
    assert np.all(np.diag(res.R) > 0)
    np.testing.assert_array_equal(np.tril(res.R, -1), 0)
    # Q spans range(A) = range(U)
    assert np.linalg.norm(res.Q - U @ (U.T @ res.Q)) < 1e-13 * kappa + 1e-12
    # R against the exact R of A = U (Sigma V^T), Sigma V^T = Q1 R0
    if kappa <= 1e8:
        _, R0 = np.linalg.qr(sig[:, None] * V.T)
        R0 = R0 * np.sign(np.diag(R0))[:, None]
        assert np.linalg.norm(res.R - R0) / np.linalg.norm(R0) < 100 * kappa * O.U_FP64 * n


def test_mrcqr_exact_factors():
    # A = U R0 with orthonormal U and upper R0 (positive diagonal) is its own QR
    U = inputs.orthonormal_matrix(2048, 20, seed=4)
    # R0 = diag(d) (I + 0.1 N), d graded 1 .. 1e-6: kappa(R0) ~ 1e6
    N = inputs.upper_with_positive_diag(20, 1.0, seed=4)
    d = np.exp(-np.log(1e6) * np.arange(20) / 19)
    R0 = d[:, None] * (np.eye(20) + 0.1 * np.triu(N, 1))
    kappa = O.cond2(R0)
    res = O.mrcqr(U @ R0, seed=1)
    # QR perturbation theory: forward errors O(kappa u)
    assert np.abs(res.Q - U).max() < 100 * kappa * O.U_FP64
    assert np.linalg.norm(res.R - R0) / np.linalg.norm(R0) < 100 * kappa * O.U_FP64


def test_mrcqr_stage2_reduces_to_cholqr():
    # with R_s = I Stage 2 is Algorithm 1 itself
    A = inputs.make_matrix(1024, 12, 10.0, seed=8)
    W = O.trsm_right_upper(A, np.eye(12))
    Rc = O.cholesky_upper(W.T @ W)
    Q = O.trsm_right_upper(W, Rc)
    Qc, Rcq = O.cholqr(A)
    np.testing.assert_array_equal(Q, Qc)
    np.testing.assert_array_equal(Rc, Rcq)


def test_mrcqr_invariant_to_sketch_scale():
    A = inputs.make_matrix(2048, 16, 1e6, seed=9)
    r1 = O.mrcqr(A, seed=2)
    r2 = O.mrcqr(A, seed=2, sketch_scale=3.0 * 2.0 ** -9)
    # equal in exact arithmetic; in FP64 within the forward error O(kappa u)
    tol = 100 * 1e6 * O.U_FP64
    assert np.abs(r2.Q - r1.Q).max() < tol
    assert np.linalg.norm(r2.R - r1.R) / np.linalg.norm(r1.R) < tol


@pytest.mark.parametrize("transform,prec,kappa", [("rfft", "fp64", 1e0), ("rfft", "fp64", 1e16), ("rfft", "fp32", 1e8),
                                                  ("rfft_reim", "fp64", 1e8), ("rfft_reim", "fp16", 1e4)])
def test_mrcqr_paper_transform_stability_experiment_shape(transform, prec, kappa):
    # Sec. III-B's shape (m = 2^17, n = 50) with the paper's sketch: c = 3n real-FFT bins (Sec. II-A)
    m, n = 1 << 17, 50
    A, U, sig, V = inputs.make_matrix(m, n, kappa, seed=21, return_factors=True)
    res = O.mrcqr(A, seed=0, prec=prec, s=3 * n, transform=transform)
    assert res.Y.shape == ((6 if transform == "rfft_reim" else 3) * n, n)
    assert O.orthogonality_error(res.Q)[0] <= 1e-13
    assert O.residual_error(A, res.Q, res.R)[0] <= 1e-13
    assert np.all(np.diag(res.R) > 0)
    if kappa <= 1e8:   # R against the exact R of A = U (Sigma V^T)
        _, R0 = np.linalg.qr(sig[:, None] * V.T)
        R0 = R0 * np.sign(np.diag(R0))[:, None]
        assert np.linalg.norm(res.R - R0) / np.linalg.norm(R0) < 100 * kappa * O.U_FP64 * n


@pytest.mark.parametrize("prec,kappa", [("fp16", 1e2), ("fp16", 1e4), ("bf16", 1e2), ("fp32", 1e4),
                                        ("fp32", 1e8)])
def test_reduced_precision_sketch_within_threshold(prec, kappa):
    # Sec. II-B: u_p * kappa <~ 1 keeps O(u) orthogonality
    A = inputs.make_matrix(4096, 32, kappa, seed=12)
    res = O.mrcqr(A, seed=0, prec=prec)
    assert O.orthogonality_error(res.Q)[0] <= 1e-13
    assert O.residual_error(A, res.Q, res.R)[0] <= 1e-13


@pytest.mark.parametrize("prec,kappa", [("fp16", 1e8), ("bf16", 1e6), ("fp32", 1e13)])
def test_reduced_precision_sketch_degrades_beyond_threshold(prec, kappa):
    # Fig. 1 / Sec. III-B: past the threshold orthogonality leaves O(u)
    A = inputs.make_matrix(4096, 32, kappa, seed=13)
    try:
        res = O.mrcqr(A, seed=0, prec=prec)
    except O.CholeskyBreakdown:
        return
    assert O.orthogonality_error(res.Q)[0] > 1e-13


@pytest.mark.parametrize("prec,kappa", [("fp16", 1e2), ("fp16", 1e3), ("fp32", 1e5), ("fp32", 1e6)])
def test_theorem1_bound_holds(prec, kappa):
    # Theorem 1 with E = R_hat_s - R_s, R_s from the FP64 sketch of the same S
    A = inputs.make_matrix(4096, 24, kappa, seed=14)
    ref = O.mrcqr(A, seed=5, prec="fp64")
    low = O.mrcqr(A, seed=5, prec=prec)
    Rs, Rh = ref.Rs, low.Rs
    eps = np.linalg.norm(Rh - Rs, 2) / np.linalg.norm(Rs, 2)
    kRs = O.cond2(Rs)
    assert eps * kRs < 1
    k1 = O.cond2(O.trsm_right_upper(A, Rs))
    k1h = O.cond2(O.trsm_right_upper(A, Rh))
    assert k1h <= O.theorem1_bound(k1, eps, kRs) * (1 + 1e-9)
    assert k1 < 10          # SRTT preconditioning: kappa(A R_s^-1) = O(1)


def test_theorem1_bound_hand_value_and_limits():
    # kappa(A R_s^-1) (1 + eps k)/(1 - eps k) with eps k = 0.1 * 5 = 0.5: 2 * 1.5 / 0.5 = 6
    assert O.theorem1_bound(2.0, 0.1, 5.0) == pytest.approx(6.0, rel=1e-15)
    assert O.theorem1_bound(3.0, 0.0, 1e10) == 3.0                   # eps k -> 0: the bound is kappa
    assert O.theorem1_bound(3.0, 1e-20, 1e10) == pytest.approx(3.0, rel=1e-9)
    assert O.theorem1_bound(1.0, 1.0 - 1e-12, 1.0) > 1e11              # eps k -> 1: unbounded
    assert math.isinf(O.theorem1_bound(1.0, 0.5, 2.0))                # eps k = 1: no bound
    assert O.theorem1_bound(1.0, 0.2, 2.0) == pytest.approx(1.4 / 0.6, rel=1e-15)


@pytest.mark.parametrize("t", [0.05, 0.3, 0.7, 0.95])
def test_theorem1_bound_attained(t):
    # Equality case: A = R_s = c I (kappa(A R_s^-1) = kappa(R_s) = 1) and
    # E = c diag(t, -t, 0, ...), so ||E|| / ||R_s|| = t and R_s + E = c diag(1+t, 1-t, 1, ...):
    # kappa(A (R_s + E)^-1) = (1 + t)/(1 - t), the bound with equality.  A
    # dropped factor, a wrong sign or a swapped ratio fails here.
    n, c = 6, 3.0
    Rs = c * np.eye(n)
    E = np.zeros((n, n))
    E[0, 0], E[1, 1] = c * t, -c * t
    A = inputs.make_matrix(64, n, 1.0, seed=2) @ Rs                   # A R_s^-1 orthonormal: kappa 1
    eps = np.linalg.norm(E, 2) / np.linalg.norm(Rs, 2)
    got = O.cond2(O.trsm_right_upper(A, Rs + E))
    bound = O.theorem1_bound(O.cond2(O.trsm_right_upper(A, Rs)), eps, O.cond2(Rs))
    assert got == pytest.approx((1 + t) / (1 - t), rel=1e-12)
    assert bound == pytest.approx(got, rel=1e-12)


def test_theorem1_bound_random_perturbations():
    # general R_s and E with eps kappa(R_s) < 1: the bound holds, and is
    # within a factor (1+t)^2/(1-t)^2 of the true value from below
    rng = np.random.default_rng(11)
    for trial in range(20):
        n = int(rng.integers(2, 12))
        Rs = np.triu(rng.standard_normal((n, n))) + 4 * np.eye(n)
        kRs = O.cond2(Rs)
        E = np.triu(rng.standard_normal((n, n)))
        t = rng.uniform(0.01, 0.9)
        E *= t / kRs * np.linalg.norm(Rs, 2) / np.linalg.norm(E, 2)
        eps = np.linalg.norm(E, 2) / np.linalg.norm(Rs, 2)
        A = inputs.make_matrix(200, n, 10.0 ** rng.uniform(0, 6), seed=trial)
        k1 = O.cond2(O.trsm_right_upper(A, Rs))
        k1h = O.cond2(O.trsm_right_upper(A, Rs + E))
        b = O.theorem1_bound(k1, eps, kRs)
        assert k1h <= b * (1 + 1e-10)
        assert k1h >= k1 * (1 - t) / (1 + t) * (1 - 1e-10)


def test_precision_rule_boundaries():
    assert O.precision_rule(1e4) == "fp16"
    assert O.precision_rule(1.0001e4) == "fp32"
    assert O.precision_rule(1e8) == "fp32"
    assert O.precision_rule(1e12) == "fp64"


# --- the double-double checks ---------------------------------------------------

def _exact_gram_minus_identity(Q):
    m, n = Q.shape
    F = [[Fraction(float(Q[i, j])) for j in range(n)] for i in range(m)]
    return [[sum(F[k][i] * F[k][j] for k in range(m)) - (1 if i == j else 0) for j in range(n)]
            for i in range(n)]


def test_dd_gram_is_correctly_rounded_sum():
    rng = np.random.default_rng(3)
    Q = np.linalg.qr(rng.standard_normal((40, 4)))[0]
    Q[5, 1] += 1e-9
    _, _, E = O.orthogonality_error(Q)
    ex = _exact_gram_minus_identity(Q)
    for i in range(4):
        for j in range(4):
            exact = ex[i][j]
            assert abs(Fraction(float(E[i, j])) - exact) <= abs(exact) * Fraction(2.0 ** -50) + Fraction(2.0 ** -100)


def test_dd_residual_exact_on_small_case():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 3))
    Q = rng.standard_normal((30, 3))
    R = np.triu(rng.standard_normal((3, 3)))
    fro, _ = O.residual_error(A, Q, R)
    tot = Fraction(0)
    for i in range(30):
        for j in range(3):
            r = Fraction(float(A[i, j])) - sum(Fraction(float(Q[i, k])) * Fraction(float(R[k, j]))
                                               for k in range(j + 1))
            tot += Fraction(float(r)) ** 2
    exact = math.sqrt(float(tot)) / np.linalg.norm(A)
    assert abs(fro - exact) <= 1e-14 * exact


def test_dd_dot_beats_naive_on_cancellation():
    x = np.array([1e16, 1.0, -1e16])
    y = np.array([1.0, 1.0, 1.0])
    assert O.dd_dot(x, y) == 1.0


def test_two_product_is_error_free():
    rng = np.random.default_rng(11)
    a = rng.standard_normal(200) * 2.0 ** rng.integers(-40, 40, 200)
    b = rng.standard_normal(200) * 2.0 ** rng.integers(-40, 40, 200)
    p, e = O.two_product(a, b)
    for i in range(200):
        assert Fraction(float(p[i])) + Fraction(float(e[i])) == Fraction(float(a[i])) * Fraction(float(b[i]))


def test_product_rounded_is_correctly_rounded_exact_sum():
    rng = np.random.default_rng(12)
    W = rng.standard_normal((6, 9)) * 2.0 ** rng.integers(-30, 30, (6, 9))
    X = np.triu(rng.standard_normal((9, 9)) * 2.0 ** rng.integers(-30, 30, (9, 9)))
    Q = O.product_rounded(W, X)
    for i in range(6):
        for j in range(9):
            exact = sum(Fraction(float(W[i, k])) * Fraction(float(X[k, j])) for k in range(9))
            assert Q[i, j] == float(exact)          # float(Fraction) rounds to nearest
    sub = O.product_rounded(W, X, rows=[4, 1])
    np.testing.assert_array_equal(sub, Q[[4, 1]])


def test_product_rounded_cancellation_and_integers():
    W = np.array([[1.0, 1e-20, -1.0]])
    assert O.product_rounded(W, np.ones((3, 1)))[0, 0] == 1e-20
    rng = np.random.default_rng(13)
    Wi = rng.integers(-1000, 1000, (20, 12)).astype(float)
    Xi = np.triu(rng.integers(-1000, 1000, (12, 12))).astype(float)
    np.testing.assert_array_equal(O.product_rounded(Wi, Xi), Wi @ Xi)


# --- Regime classification without learning (Sec. II-C) -------------------------

def test_regime_thresholds():
    # half below 1e4, single below 1e8, double beyond (boundaries as precision_rule)
    assert [O.regime_of(k) for k in (1.0, 1e4, 1.0001e4, 1e8, 1.0001e8, math.inf)] == [0, 0, 1, 1, 2, 2]


@pytest.mark.parametrize("n", [1, 3, 4])
def test_onenorm_estimate_exact_for_tiny_n(n):
    B = inputs.gaussian(n, n, seed=n)
    est = O.onenorm_estimate(lambda X: B @ X, lambda X: B.T @ X, n)
    assert est == pytest.approx(np.abs(B).sum(axis=0).max(), rel=1e-15)


def test_onenorm_estimate_exact_on_diagonal_and_dominant_column():
    # the estimator's second step lands on the unit vector of the largest column
    n = 50
    d = np.linspace(1.0, 3.0, n)[::-1].copy()
    np.random.default_rng(1).shuffle(d)
    B = np.diag(d)
    assert O.onenorm_estimate(lambda X: B @ X, lambda X: B.T @ X, n) == pytest.approx(d.max(), rel=1e-15)
    C = 0.01 * inputs.gaussian(n, n, seed=2)
    C[:, 17] += 5.0
    exact = np.abs(C).sum(axis=0).max()
    assert O.onenorm_estimate(lambda X: C @ X, lambda X: C.T @ X, n) == pytest.approx(exact, rel=1e-14)


def test_onenorm_estimate_lower_bound_and_close():
    # est = ||B x||_1 for some ||x||_1 = 1, so est <= ||B||_1; Higham and Tisseur report it within a
    # small factor, usually exact; scipy's implementation of the same algorithm (its own random
    # columns) is the library cross-check
    import scipy.sparse.linalg as sl
    rng = np.random.default_rng(0)
    ratios, scipy_ratios = [], []
    for trial in range(40):
        n = int(rng.integers(5, 80))
        B = rng.standard_normal((n, n))
        exact = np.abs(B).sum(axis=0).max()
        est = O.onenorm_estimate(lambda X: B @ X, lambda X: B.T @ X, n, seed=trial)
        assert est <= exact * (1 + 1e-12)
        ratios.append(est / exact)
        scipy_ratios.append(sl.onenormest(B) / exact)
    assert min(ratios) > 0.5 and np.mean(ratios) > 0.85
    assert abs(np.mean(ratios) - np.mean(scipy_ratios)) < 0.1


@pytest.mark.parametrize("kappa", [1e0, 1e2, 1e4, 1e6, 1e7])
def test_cholqr_probe_is_a_lower_bound(kappa):
    # Sec. II-C: kappa_2(A) >= sqrt(q / (u (1 + q))), q = ||I - Q^T Q||_2 of CholQR
    A = inputs.make_matrix(4096, 32, kappa, seed=3)
    est, q = O.cholqr_probe(A)
    k2 = O.cond2(A)
    if kappa >= 1e2:   # once CholQR's loss of orthogonality exceeds the rounding floor
        assert k2 / 100 <= est <= k2
    else:              # at kappa ~ 1, q sits on the floor of a few u: the value is O(1)
        assert q < 32 * O.U_FP64 and est < 8
    assert O.cholqr_probe(inputs.make_matrix(4096, 32, 1e10, seed=3))[0] == math.inf   # breakdown


@pytest.mark.parametrize("kappa", [1e0, 1e3, 1e6])
def test_onenorm_regime_estimate_brackets_kappa(kappa):
    # kappa_2^2 <= n ||G||_1 ||G^-1||_1 <= n^2 kappa_2^2 with the exact norm; the estimate of
    # ||G^-1||_1 is a lower bound within a small factor of it
    m, n = 4096, 24
    A = inputs.make_matrix(m, n, kappa, seed=5)
    est, g1, ginv1 = O.onenorm_regime_estimate(A)
    G = A.T @ A
    exact = np.abs(np.linalg.inv(G)).sum(axis=0).max()
    assert g1 == pytest.approx(np.abs(G).sum(axis=0).max(), rel=1e-15)
    assert ginv1 <= exact * (1 + 1e-8) and ginv1 >= exact / 3
    k2 = O.cond2(A)
    assert est >= k2 / 2 and est <= n * k2 * (1 + 1e-8)
    assert O.onenorm_regime_estimate(inputs.make_matrix(m, n, 1e10, seed=5))[0] == math.inf


# --- Small definitions the sketches and the estimator rest on --------------------

def test_seed_key_splits_the_64_bit_seed():
    # key = (low word, high word) of the seed, so seed = k0 + 2^32 k1
    assert O.seed_key(0) == (0, 0)
    assert O.seed_key(2 ** 40 + 5) == (5, 256)
    assert O.seed_key(2 ** 64 - 1) == (2 ** 32 - 1, 2 ** 32 - 1)


def test_column_scale_exponents_place_the_maximum_in_the_fp16_window():
    # max_i |a_ij| 2^e_j in [2^13, 2^14) (keeps the FP16 sketch clear of underflow); zero columns keep 0
    rng = np.random.default_rng(3)
    A = rng.standard_normal((64, 6)) * np.array([1e-30, 1e-5, 1.0, 3.0, 1e12, 0.0])
    A[0, 2] = 2.0 ** 13                # an exact power of two: e = 0
    e = O.column_scale_exponents(A)
    scaled = np.abs(np.ldexp(A, e[None, :])).max(axis=0)
    assert np.all((scaled[:5] >= 2.0 ** 13) & (scaled[:5] < 2.0 ** 14))
    assert e[2] == 0 and e[5] == 0


def test_random_sign_columns_of_the_estimator():
    # +-1 entries from Philox at counter (i, 2, draw, 0): deterministic, balanced, distinct across draws
    a = O.random_sign_column(4096, seed=11, draw=0)
    assert set(np.unique(a)) == {-1.0, 1.0}
    np.testing.assert_array_equal(a, O.random_sign_column(4096, seed=11, draw=0))
    assert abs(a.sum()) <= 5 * math.sqrt(4096)
    b = O.random_sign_column(4096, seed=11, draw=1)
    assert abs(float(a @ b)) < 4096 / 4          # a new draw is not (anti-)parallel
    # the counter's second word separates it from the Rademacher signs (word 0 of counter (i, 0, 0, 0))
    assert not np.array_equal(a, O.rademacher(4096, 11))
