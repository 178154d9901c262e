"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: signs and sample indices.  Floating point: the parity bounds
-- sketch within 5e-3 (FP16/BF16), 1e-5 (FP32) relative Frobenius of the FP64
oracle sketch (1e-13 for the FP64 sketch: same arithmetic, different
summation order); ||I - Q^T Q||_2 <= 1e-13 and ||A - QR||_F / ||A||_F <= 1e-13
at the precision the paper's bounds allow (Sec. II-B)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu

SKETCH_TOL = {"fp16": 5e-3, "bf16": 5e-3, "fp32": 1e-5, "fp64": 1e-13}


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_18411_gb300 import build
    build.build()
    from paper_2606_18411_gb300 import mrcqr
    return mrcqr


def _np(t):
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --- Algorithm 2 step 1 ------------------------------------------------------

@pytest.mark.parametrize("m,seed", [(1, 0), (4097, 0), (1 << 20, 7), ((1 << 22) + 3, 2 ** 40 + 5)])
def test_signs_bit_exact(M, m, seed):
    np.testing.assert_array_equal(_np(M.signs(m, seed)), O.rademacher(m, seed))


@pytest.mark.parametrize("m,s,seed", [(1, 1, 0), (64, 64, 3), (4096, 64, 0), (4096 + 17, 66, 9),
                                      (1 << 20, 256, 1), (1 << 22, 1024, 12345), (300000, 8192, 2 ** 33 + 1)])
def test_sample_rows_bit_exact(M, m, s, seed):
    got = _np(M.sample_rows(m, s, seed)).astype(np.int64)
    np.testing.assert_array_equal(got, O.sample_rows(m, s, seed))


def test_fl_p_bit_exact(M):
    import torch
    rng = np.random.default_rng(7)
    x = rng.standard_normal(200000) * np.exp2(rng.integers(-40, 20, 200000))
    x = np.concatenate([x, [0.0, -0.0, 65504.0, 65519.9, 65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26,
                            1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, 2.0 ** -1030, -(2.0 ** -1074)]])
    xd = torch.from_numpy(x).cuda()
    # FP16 and FP32: numpy's correctly rounded casts (normal and subnormal range)
    np.testing.assert_array_equal(_np(M.round_to("fp16", xd)), x.astype(np.float16).astype(np.float64))
    y = rng.standard_normal(200000) * np.exp2(rng.integers(-160, 120, 200000))
    np.testing.assert_array_equal(_np(M.round_to("fp32", torch.from_numpy(y).cuda())),
                                  y.astype(np.float32).astype(np.float64))
    # BF16: the oracle's significand rounding in the normal range
    z = rng.standard_normal(200000) * np.exp2(rng.integers(-100, 100, 200000))
    np.testing.assert_array_equal(_np(M.round_to("bf16", torch.from_numpy(z).cuda())), O.round_significand(z, 8))


# --- Algorithm 2 steps 2-4 -------------------------------------------------------

@pytest.mark.parametrize("m", [8, 64, 256])
def test_sketch_brute_force_tiny(M, m):
    # s = m: every row of S sampled; elementwise against the dense S A
    n = 5
    A = inputs.gaussian(m, n, seed=m)
    Y = _np(M.sketch(M.to_colmajor(A), m, "fp64", seed=3))
    ref = O.sketch(A, O.sample_rows(m, m, 3), O.rademacher(m, 3))
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32", "fp64"])
@pytest.mark.parametrize("m,n", [(4096, 32), (4096 + 17, 33), (20000, 100), (1000, 7)])
def test_sketch_against_oracle(M, prec, m, n):
    s = 2 * n
    A = inputs.make_matrix(m, n, 1e8, seed=m + n)
    Y = _np(M.sketch(M.to_colmajor(A), s, prec, seed=11))
    d, idx = O.rademacher(m, 11), O.sample_rows(m, s, 11)
    ref = O.sketch(A, idx, d)
    err = _rel(Y, ref)
    assert err <= SKETCH_TOL[prec], err
    if prec != "fp64":
        # the fl_p error model of the oracle agrees within the same order
        emu = O.sketch_emulated(A, idx, d, prec)
        assert _rel(Y, emu) <= 2 * SKETCH_TOL[prec]


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("m,n", [(4096, 32), (4096 + 18, 33), (20000, 100), (1000, 7), (1 << 16, 128),
                                 (30000, 200)])
def test_sketch_tensor_core_against_oracle(M, prec, m, n):
    # tcgen05 variant (A 16-byte aligned, lda even); ragged m, n and s = 2n
    s = 2 * n
    A = inputs.make_matrix(m, n, 1e6, seed=m + 3 * n)
    Y = _np(M.sketch(M.to_colmajor(A), s, prec, seed=17, variant=2))
    assert M.last_sketch_variant() == 2
    d, idx = O.rademacher(m, 17), O.sample_rows(m, s, 17)
    ref = O.sketch(A, idx, d)
    err = _rel(Y, ref)
    assert err <= SKETCH_TOL[prec], err
    emu = O.sketch_emulated(A, idx, d, prec)
    assert _rel(Y, emu) <= 2 * SKETCH_TOL[prec]


def test_sketch_variants_agree_and_fall_back(M):
    m, n = 8192, 48
    A = inputs.make_matrix(m, n, 1e3, seed=9)
    Ad = M.to_colmajor(A)
    y_tc = _np(M.sketch(Ad, 2 * n, "fp16", seed=5, variant=2))
    assert M.last_sketch_variant() == 2
    y_simt = _np(M.sketch(Ad, 2 * n, "fp16", seed=5, variant=1))
    assert M.last_sketch_variant() == 1
    assert _rel(y_tc, y_simt) < 5e-3
    # odd leading dimension: no TMA map; the tensor-core kernel stages A with plain copies
    Aodd = M.to_colmajor(A, ld=m + 1)
    y_odd = _np(M.sketch(Aodd, 2 * n, "fp16", seed=5))
    assert M.last_sketch_variant() == 2
    np.testing.assert_array_equal(y_odd, y_tc)
    # FP64: emulated FP64 on the tensor cores (from digit planes) unless the SIMT variant is asked for
    _ = M.sketch(Ad, 2 * n, "fp64", seed=5, variant=2)
    assert M.last_sketch_variant() == 5
    _ = M.sketch(Ad, 2 * n, "fp64", seed=5)
    assert M.last_sketch_variant() == 5
    _ = M.sketch(Ad, 2 * n, "fp64", seed=5, variant=1)
    assert M.last_sketch_variant() == 1


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("m,n,s", [(2048, 5, 30), (3072, 7, 14), (8192, 33, 66), (1 << 16, 128, 256),
                                   (5 << 13, 100, 200), (1 << 15, 3, 1024), (1 << 17, 64, 128)])
def test_sketch_four_step_against_oracle(M, prec, m, n, s):
    # the four-step variant (radix-64 DFT of the strided subsequences on the tensor cores, then only
    # the s sampled outputs): m a multiple of 1024 (power of two or not), ragged n, s up to 1024
    A = inputs.make_matrix(m, n, 1e6, seed=m + 5 * n)
    Y = _np(M.sketch(M.to_colmajor(A), s, prec, seed=19, variant=4))
    assert M.last_sketch_variant() == 4
    d, idx = O.rademacher(m, 19), O.sample_rows(m, s, 19)
    ref = O.sketch(A, idx, d)
    assert _rel(Y, ref) <= SKETCH_TOL[prec], _rel(Y, ref)
    emu = O.sketch_emulated(A, idx, d, prec)
    assert _rel(Y, emu) <= 2 * SKETCH_TOL[prec]
    # per column as well (the 2^e scale is per tile and column)
    colerr = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert colerr.max() <= 2 * SKETCH_TOL[prec]


def test_sketch_four_step_falls_back(M):
    # not a multiple of 1024 rows, or the real-FFT transform: the dense-row tensor-core variant runs
    A = inputs.make_matrix(5000, 16, 1e3, seed=3)
    _ = M.sketch(M.to_colmajor(A), 32, "fp16", seed=1, variant=4)
    assert M.last_sketch_variant() == 2
    B = M.to_colmajor(inputs.make_matrix(4096, 16, 1e3, seed=4))
    _ = M.sketch_transform(B, 32, "rfft", prec="fp16", seed=1, variant=4)
    assert M.last_sketch_variant() == 2
    # odd leading dimension: no TMA map, so no four-step; the dense-row kernel copies A without TMA
    _ = M.sketch(M.to_colmajor(inputs.make_matrix(4096, 16, 1e3, seed=5), ld=4097), 32, "fp16", seed=1, variant=4)
    assert M.last_sketch_variant() == 2


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("m,n,ld", [(5001, 70, 5001), (4096, 130, 4097), (777, 3, 779), (40000, 64, 40001)])
def test_sketch_plain_copies_match_tma(M, prec, m, n, ld):
    # the same matrix once with a TMA-describable layout (even ld) and once without (odd ld):
    # the two staging paths feed identical tiles to the same arithmetic, so Y is bit for bit the same
    A = inputs.make_matrix(m, n, 1e4, seed=m + n)
    s = 2 * n
    ld_even = ld + 1 if ld % 2 else ld
    y_tma = _np(M.sketch(M.to_colmajor(A, ld=ld_even), s, prec, seed=23, variant=2))
    assert M.last_sketch_variant() == 2
    y_plain = _np(M.sketch(M.to_colmajor(A, ld=ld), s, prec, seed=23, variant=2))
    assert M.last_sketch_variant() == 2
    np.testing.assert_array_equal(y_plain, y_tma)
    d, idx = O.rademacher(m, 23), O.sample_rows(m, s, 23)
    assert _rel(y_plain, O.sketch(A, idx, d)) <= SKETCH_TOL[prec]


def test_sketch_scale_exponent_keeps_fp16_in_range(M):
    # columns of very different magnitude (1e-12 .. 1e6): per-column 2^e scaling
    m, n = 8192, 8
    A = inputs.gaussian(m, n, seed=5) * np.logspace(-12, 6, n)[None, :]
    Y = _np(M.sketch(M.to_colmajor(A), 16, "fp16", seed=1))
    ref = O.sketch(A, O.sample_rows(m, 16, 1), O.rademacher(m, 1))
    colerr = np.linalg.norm(Y - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert colerr.max() < 5e-3


# --- Algorithm 2 steps 5-6 -------------------------------------------------------

@pytest.mark.parametrize("prec,n", [("fp64", 32), ("fp64", 100), ("fp32", 32), ("fp32", 129)])
def test_sketch_qr_against_householder(M, prec, n):
    s = 2 * n
    Y = inputs.gaussian(s, n, seed=n) * np.logspace(0, -6, n)[None, :]
    Rs = _np(M.sketch_qr(M.to_colmajor(Y), prec))
    ref = O.householder_qr(Y)
    assert np.all(np.diag(Rs) > 0)
    np.testing.assert_array_equal(np.tril(Rs, -1), 0)
    # column-scaled Gaussian: Householder errors are columnwise ~ u_p
    tol = 1e-12 if prec == "fp64" else 1e-4
    colerr = np.linalg.norm(Rs - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert colerr.max() < tol


# --- Algorithm 1 / Algorithm 2 steps 7-9 -----------------------------------------

def test_stage2_with_identity_is_cholqr(M):
    A = inputs.make_matrix(20000, 24, 100.0, seed=3)
    Q, R = M.cholqr_precond(M.to_colmajor(A), M.to_colmajor(np.eye(24)))
    Qr, Rr = O.cholqr(A)
    np.testing.assert_allclose(_np(R), Rr, rtol=0, atol=1e-12 * np.abs(Rr).max())
    np.testing.assert_allclose(_np(Q), Qr, rtol=0, atol=1e-12)


def test_stage2_orthonormal_input(M):
    U = inputs.orthonormal_matrix(50000, 40, seed=2)
    Q, R = M.cholqr_precond(M.to_colmajor(U), M.to_colmajor(np.eye(40)))
    np.testing.assert_allclose(_np(Q), U, atol=1e-14)
    np.testing.assert_allclose(_np(R), np.eye(40), atol=1e-14)


def test_stage2_given_preconditioner_matches_oracle(M):
    A = inputs.make_matrix(30000, 48, 1e12, seed=4)
    ref = O.mrcqr(A, seed=1, prec="fp64")
    Q, R = M.cholqr_precond(M.to_colmajor(A), M.to_colmajor(ref.Rs))
    assert M.last_status()["status"] == "OK"
    Qh, Rh = _np(Q), _np(R)
    assert O.orthogonality_error(Qh)[0] <= 1e-13
    assert O.residual_error(A, Qh, Rh)[0] <= 1e-13
    # same R_s, same arithmetic up to summation order: W and R_c agree to ~u kappa(W)
    assert _rel(Rh, ref.R) < 1e-10


# --- Algorithm 2 end to end ------------------------------------------------------

def _check_factor(M, A, prec, seed=0, expect_prec=None, **kw):
    Ad = M.to_colmajor(A)
    Q, R = M.factor(Ad, prec=prec, seed=seed, **kw)
    st = M.last_status()
    Qh, Rh = _np(Q), _np(R)
    o2, of, _ = O.orthogonality_error(Qh)
    rf, r2 = O.residual_error(A, Qh, Rh)
    return st, o2, rf, Qh, Rh


@pytest.mark.parametrize("kappa", [1e0, 1e4, 1e7])
def test_cholqr2_against_oracle(M, kappa):
    # the stability experiment's comparison method: O(u) while kappa^2 u < 1
    A = inputs.make_matrix(8193, 48, kappa, seed=17)
    Q, R = M.cholqr2(M.to_colmajor(A))
    st = M.last_status()
    Qh, Rh = _np(Q), _np(R)
    assert st["status"] == "OK", st
    o2 = O.orthogonality_error(Qh)[0]
    rf = O.residual_error(A, Qh, Rh)[0]
    assert o2 <= 1e-13 and rf <= 1e-13, (o2, rf)
    Qo, Ro = O.cholqr2(A)
    assert _rel(Rh, Ro) < 100 * kappa * O.U_FP64
    np.testing.assert_array_equal(np.tril(Rh, -1), 0)


def test_cholqr2_breaks_down_past_1e8(M):
    A = inputs.make_matrix(8193, 48, 1e12, seed=18)
    M.cholqr2(M.to_colmajor(A))
    assert M.last_status()["status"] in ("BREAKDOWN", "ORTHO")


def test_config1_fp32_sketch(M):
    # m=4096, n=32, geometric sigma 1..1e-8, FP32 sketch, s=2n, seed 0
    A = inputs.make_matrix(4096, 32, 1e8, seed=1001)
    st, o2, rf, Qh, Rh = _check_factor(M, A, "fp32", seed=0)
    assert st["status"] == "OK" and st["retries"] == 0 and st["prec_used"] == "fp32"
    assert o2 <= 1e-13 and rf <= 1e-13
    assert np.all(np.diag(Rh) > 0)
    np.testing.assert_array_equal(np.tril(Rh, -1), 0)
    ref = O.mrcqr(A, seed=0, prec="fp32")
    # two backward-stable QRs of the same A with diag(R) > 0: forward error O(kappa u)
    assert _rel(Rh, ref.R) < 1e4 * 1e8 * O.U_FP64
    assert st["ortho_fro"] <= 1e-13


@pytest.mark.parametrize("kappa", [1e0, 1e2, 1e4, 1e8, 1e12, 1e16])
@pytest.mark.parametrize("m,n", [(4096, 16), (10007, 50), (16384, 128)])
def test_rule_precision_end_to_end(M, kappa, m, n):
    prec = O.precision_rule(kappa)
    A = inputs.make_matrix(m, n, kappa, seed=int(np.log10(kappa)) + 7 * n)
    st, o2, rf, _, _ = _check_factor(M, A, prec, seed=3)
    assert st["status"] == "OK", st
    assert o2 <= 1e-13 and rf <= 1e-13, (o2, rf)


# Edge shapes: one column; the smallest legal m (m = s = 2n, every row of the
# transform sampled); the widest n at a small ragged m.  Checked in
# double-double, and R against the oracle's R: two backward-stable QRs of the
# same A with diag(R) > 0 differ by O(kappa u) (the thin QR with a positive
# diagonal is unique).
@pytest.mark.parametrize("m,n,kappa", [(2, 1, 1.0), (4097, 1, 1.0), (64, 32, 1e4), (256, 128, 1e8),
                                       (1024, 512, 1e2), (1031, 512, 1e8), (1031, 512, 1e12), (1030, 509, 1e6)])
def test_edge_shapes_against_oracle(M, m, n, kappa):
    prec = O.precision_rule(kappa)
    A = inputs.make_matrix(m, n, kappa, seed=31 + m + n)
    st, o2, rf, Qh, Rh = _check_factor(M, A, prec, seed=6)
    assert st["status"] == "OK", st
    assert o2 <= 1e-13 and rf <= 1e-13, (o2, rf)
    assert np.all(np.diag(Rh) > 0)
    np.testing.assert_array_equal(np.tril(Rh, -1), 0)
    if kappa <= 1e8:
        ref = O.mrcqr(A, seed=6, prec=st["prec_used"])
        assert _rel(Rh, ref.R) <= 100 * kappa * O.U_FP64, _rel(Rh, ref.R)
        # and against a plain Householder QR of A (the exact-definition check)
        assert _rel(Rh, O.householder_qr(A)) <= 100 * kappa * O.U_FP64


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e8])
def test_r_against_oracle_at_rule_precision(M, kappa):
    # R against the oracle's R (same seed, same sketch precision) and the
    # oracle's Householder R at C kappa u, ragged m and n
    m, n = 20011, 96
    prec = O.precision_rule(kappa)
    A = inputs.make_matrix(m, n, kappa, seed=41)
    st, o2, rf, Qh, Rh = _check_factor(M, A, prec, seed=8)
    assert st["status"] == "OK" and st["retries"] == 0, st
    ref = O.mrcqr(A, seed=8, prec=prec)
    assert _rel(Rh, ref.R) <= 100 * kappa * O.U_FP64
    assert _rel(Rh, O.householder_qr(A)) <= 100 * kappa * O.U_FP64
    # Q against the oracle's Q: the same O(kappa u) forward error
    assert _rel(Qh, ref.Q) <= 100 * kappa * O.U_FP64


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_escalation_on_underestimated_precision(M, prec):
    # Sec. II-C: a too-low precision is detected and re-run higher
    A = inputs.make_matrix(8192, 32, 1e13, seed=21)
    st, o2, rf, _, _ = _check_factor(M, A, prec, seed=2)
    assert st["status"] == "OK" and st["retries"] >= 1 and st["prec_used"] == "fp64"
    assert o2 <= 1e-13 and rf <= 1e-13


def test_no_escalation_reports_failure(M):
    A = inputs.make_matrix(8192, 32, 1e12, seed=22)
    Ad = M.to_colmajor(A)
    Q = M.empty_colmajor(8192, 32)
    R = M.empty_colmajor(32, 32)
    M.factor_ex(Ad, Q, R, prec="fp16", seed=0, escalate=False)
    st = M.last_status()
    assert st["status"] in ("ORTHO", "BREAKDOWN") and st["retries"] == 0


def test_nonfinite_input(M):
    A = inputs.make_matrix(4096, 16, 10.0, seed=23)
    A[100, 3] = np.nan
    _, _ = M.factor(M.to_colmajor(A), prec="fp32")
    assert M.last_status()["status"] == "NONFINITE"


def test_rank_deficient_input(M):
    # column 9 repeats column 5: either the run is flagged (breakdown / failed
    # check), or it returns a valid thin QR of the singular A whose R shows the
    # rank deficiency (R[9, 9] at rounding level)
    A = inputs.make_matrix(4096, 16, 10.0, seed=24)
    A[:, 9] = A[:, 5]
    Q, R = M.factor(M.to_colmajor(A), prec="fp64")
    st = M.last_status()
    assert st["status"] in ("OK", "BREAKDOWN", "ORTHO")
    if st["status"] == "OK":
        Qh, Rh = _np(Q), _np(R)
        assert O.orthogonality_error(Qh)[0] <= 1e-13
        assert O.residual_error(A, Qh, Rh)[0] <= 1e-13
        assert abs(Rh[9, 9]) <= 1e-12 * np.linalg.norm(Rh)


def test_deterministic(M):
    A = M.to_colmajor(inputs.make_matrix(50000, 64, 1e8, seed=25))
    Q1, R1 = M.factor(A, prec="fp32", seed=4)
    Q2, R2 = M.factor(A, prec="fp32", seed=4)
    assert (Q1 == Q2).all().item() and (R1 == R2).all().item()


def test_leading_dimensions(M):
    m, n = 5000, 20
    A = inputs.make_matrix(m, n, 1e6, seed=26)
    Ad = M.to_colmajor(A, ld=m + 13)
    Q = M.empty_colmajor(m, n, ld=m + 5)
    import torch
    Rbig = torch.zeros((n, n + 3), dtype=torch.float64, device="cuda").t()[:n]
    M.factor_ex(Ad, Q, Rbig, prec="fp32", seed=1)
    assert M.last_status()["status"] == "OK"
    Qh, Rh = _np(Q), _np(Rbig)
    assert O.orthogonality_error(Qh)[0] <= 1e-13 and O.residual_error(A, Qh, Rh)[0] <= 1e-13


def test_bounded_wait_reports_timeout_and_context_survives(M):
    # a wait on a barrier that nothing completes gives up after its bound and reports TIMEOUT
    # (no fault, trap or endless loop); the context then still runs a factorization
    import torch
    from paper_2606_18411_gb300 import _lib
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert _lib.load().mrcqr_debug_wait_timeout(4096, status.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 7                       # MRCQR_ERR_TIMEOUT
    A = inputs.make_matrix(4096, 16, 1e3, seed=1)
    Q, R = M.factor(M.to_colmajor(A), prec="fp16")
    torch.cuda.synchronize()
    assert M.last_status()["status"] == "OK"
    assert O.orthogonality_error(Q.cpu().numpy())[0] <= 1e-13
