"""The paper's own sketch transform (Algorithm 2 as printed, Sec. II-A) on the
CUDA path, against the oracle: the real parts of c sampled bins of the real
FFT of D A (scale sqrt(c/m)), and the variant that stacks their imaginary
parts below (a 2c x n sketch).

Bit-exact: the sampled bins.  Floating point: the sketch within the bounds of
the DCT sketch tests (5e-3 FP16/BF16, 1e-5 FP32, 1e-13 FP64, relative
Frobenius against the FP64 oracle); end to end ||I - Q^T Q||_2 <= 1e-13 and
||A - QR||_F / ||A||_F <= 1e-13 at the stability experiment's shape
(m = 2^17, n = 50, c = 3n; Sec. III-B)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu

SKETCH_TOL = {"fp16": 5e-3, "bf16": 5e-3, "fp32": 1e-5, "fp64": 1e-13}
IM = np.uint32(0x80000000)


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


def _oracle_sketch(A, c, seed, transform, prec="fp64"):
    m = A.shape[0]
    d, bins = O.rademacher(m, seed), O.sample_bins(m, c, seed)
    imag = transform == "rfft_reim"
    if prec == "fp64":
        return O.rfft_sketch(A, bins, d, imag=imag)
    return O.rfft_sketch_emulated(A, bins, d, prec, imag=imag)


# --- Algorithm 2 step 1: bins of the real FFT ---------------------------------

@pytest.mark.parametrize("m,c,seed", [(1, 1, 0), (2, 2, 0), (7, 4, 3), (64, 33, 1), (4096, 150, 0),
                                      (1 << 17, 150, 0), ((1 << 20) + 3, 384, 7), (300001, 4096, 2 ** 33 + 1)])
@pytest.mark.parametrize("transform", ["rfft", "rfft_reim"])
def test_sample_bins_bit_exact(M, m, c, seed, transform):
    if transform == "rfft_reim" and 2 * c > 8192:
        pytest.skip("2c rows above the sketch limit")
    got = _np(M.sample_transform_rows(m, c, transform, seed)).view(np.uint32)
    ref = O.sample_bins(m, c, seed).astype(np.uint32)
    np.testing.assert_array_equal(got[:c], ref)
    if transform == "rfft_reim":
        np.testing.assert_array_equal(got[c:], ref | IM)     # the Im rows of the same bins


def test_sample_rows_dct_unchanged(M):
    # the DCT transform draws from {0..m-1} exactly as mrcqr_sample_rows
    got = _np(M.sample_transform_rows(4097, 66, "dct", 9)).astype(np.int64)
    np.testing.assert_array_equal(got, O.sample_rows(4097, 66, 9))


def test_sample_bins_rejects_more_bins_than_the_spectrum(M):
    from paper_2606_18411_gb300 import _lib
    import torch
    idx = torch.empty(64, dtype=torch.int32, device="cuda")
    lib = _lib.load()
    assert lib.mrcqr_sample_transform_rows(100, 52, 1, 0, idx.data_ptr(), None) == 1   # 51 bins
    assert lib.mrcqr_sample_transform_rows(100, 51, 1, 0, idx.data_ptr(), None) == 0
    assert lib.mrcqr_sample_transform_rows(100, 51, 3, 0, idx.data_ptr(), None) == 1   # no such transform


# --- Algorithm 2 steps 2-4 ------------------------------------------------------

@pytest.mark.parametrize("m", [8, 9, 64, 257])
@pytest.mark.parametrize("transform", ["rfft", "rfft_reim"])
def test_sketch_all_bins_brute_force(M, m, transform):
    # every bin sampled (c = floor(m/2) + 1), elementwise against the dense rows of S
    n, c = 5, m // 2 + 1
    A = inputs.gaussian(m, n, seed=m)
    Y = _np(M.sketch_transform(M.to_colmajor(A), c, transform, "fp64", seed=3))
    ref = _oracle_sketch(A, c, 3, transform)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32", "fp64"])
@pytest.mark.parametrize("transform", ["rfft", "rfft_reim"])
@pytest.mark.parametrize("m,n", [(4096, 32), (4096 + 18, 33), (20000, 100), (1 << 17, 50)])
def test_sketch_against_oracle(M, m, n, transform, prec, variant):
    # SIMT (variant 1) and tensor-core (variant 2; emulated FP64 for fp64) kernels, c = 3n
    c = 3 * n
    A = inputs.make_matrix(m, n, 1e8, seed=m + n)
    Y = _np(M.sketch_transform(M.to_colmajor(A), c, transform, prec, seed=11, variant=variant))
    assert Y.shape == ((2 if transform == "rfft_reim" else 1) * c, n)
    ref = _oracle_sketch(A, c, 11, transform)
    err = _rel(Y, ref)
    assert err <= SKETCH_TOL[prec], err
    if prec != "fp64":
        # the oracle's fl_p error model agrees within the same order
        assert _rel(Y, _oracle_sketch(A, c, 11, transform, prec)) <= 2 * SKETCH_TOL[prec]


# --- Algorithm 2 end to end ---------------------------------------------------------

def _factor(M, A, prec, transform, s_factor=3, escalate=True):
    import torch
    from paper_2606_18411_gb300 import _lib
    m, n = A.shape
    Q = M.empty_colmajor(m, n, device=A.device)
    R = M.empty_colmajor(n, n, device=A.device)
    stats = torch.zeros(8, dtype=torch.float64, device=A.device)
    M.factor_ex(A, Q, R, prec=prec, seed=0, s_factor=s_factor, escalate=escalate, transform=transform,
                stats_device=stats)
    torch.cuda.synchronize()
    return Q, R, _lib.Stats.from_buffer_copy(stats.cpu().numpy().tobytes()).as_dict()


@pytest.mark.parametrize("kappa", [1e0, 1e4, 1e8, 1e12, 1e16])
@pytest.mark.parametrize("transform", ["rfft", "rfft_reim"])
def test_paper_transform_stability_experiment_shape(M, transform, kappa):
    # Sec. III-B's shape with the paper's sketch, c = 3n bins, precision by the regime rule
    m, n = 1 << 17, 50
    prec = O.precision_rule(kappa)
    A, U, sig, V = inputs.make_matrix(m, n, kappa, seed=21, return_factors=True)
    Q, R, st = _factor(M, M.to_colmajor(A), prec, transform)
    assert st["status"] == "OK" and st["ortho_fro"] <= 1e-13, st
    Qh, Rh = _np(Q), _np(R)
    assert O.orthogonality_error(Qh)[0] <= 1e-13
    assert O.residual_error(A, Qh, Rh)[0] <= 1e-13
    assert np.all(np.diag(Rh) > 0) and np.all(np.tril(Rh, -1) == 0)
    if kappa <= 1e8:   # R is unique: against the exact R of A = U (Sigma V^T)
        _, R0 = np.linalg.qr(sig[:, None] * V.T)
        R0 = R0 * np.sign(np.diag(R0))[:, None]
        assert np.linalg.norm(Rh - R0) / np.linalg.norm(R0) < 100 * kappa * O.U_FP64 * n


@pytest.mark.parametrize("transform", ["rfft", "rfft_reim"])
def test_paper_transform_matches_oracle_preconditioner(M, transform):
    # the FP64 sketch's R_s through the C ABI against the oracle's (same bins and signs)
    m, n = 20000, 24
    A = inputs.make_matrix(m, n, 1e10, seed=5)
    Y = M.sketch_transform(M.to_colmajor(A), 3 * n, transform, "fp64", seed=0)
    Rs = _np(M.sketch_qr(Y, "fp64"))
    ref = O.householder_qr(_oracle_sketch(A, 3 * n, 0, transform))
    assert np.linalg.norm(Rs - ref) / np.linalg.norm(ref) < 1e-12


def test_paper_transform_without_escalation_fails_far_outside_the_regime(M):
    # FP16 real-FFT sketch at kappa = 1e12 cannot reach the bound (Sec. II-B) and says so
    m, n = 1 << 16, 32
    A = inputs.make_matrix(m, n, 1e12, seed=3)
    _, _, st = _factor(M, M.to_colmajor(A), "fp16", "rfft", escalate=False)
    assert st["status"] != "OK"
    _, _, st = _factor(M, M.to_colmajor(A), "fp16", "rfft", escalate=True)
    assert st["status"] == "OK" and st["retries"] >= 1


def test_reim_rejects_more_than_8192_rows(M):
    import torch
    m, n = 1 << 16, 512
    A = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    Q = M.empty_colmajor(m, n, device="cuda")
    R = M.empty_colmajor(n, n, device="cuda")
    with pytest.raises(RuntimeError):
        M.factor_ex(A, Q, R, prec="fp64", s_factor=9, transform="rfft_reim")   # 2 x 9 x 512 rows
