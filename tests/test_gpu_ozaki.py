"""Emulated FP64 products on the FP16 tensor cores (exact digit slicing)
against the correctly rounded exact product of the oracle, and the full
factorization with and without them."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_18411_gb300 import build
    build.build()
    from paper_2606_18411_gb300 import mrcqr as M
    return torch, M


def _operands(m, n, seed, graded=False):
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((m, n)) / np.sqrt(m)
    if graded:                                   # rows and columns over many binades
        W *= 2.0 ** rng.integers(-30, 30, (m, 1))
        W *= 2.0 ** rng.integers(-8, 8, (1, n))
    X = np.triu(rng.standard_normal((n, n)) * 0.05) + np.diag(1.0 + rng.random(n))
    if graded:
        X *= 2.0 ** rng.integers(-20, 20, (1, n))
    return W, X


def _run(env, W, X, fp64_products):
    torch, M = env
    Wd = M.to_colmajor(W)
    Xd = M.to_colmajor(X)
    M.finalize_q(Wd, Xd, fp64_products=fp64_products)
    torch.cuda.synchronize()
    return Wd.cpu().numpy()


def _bounds(W, X, rows):
    """Per-entry bounds against the correctly rounded exact value (one more
    half ulp, <= u |exact|, than against the exact sum): emulated
    |err| <= 2u|exact| + 2^-57 (j+1) R_i C_j (a once-rounded value of a sum
    that is off by the slicing error), FP64 FMA |err| <= u|exact| +
    gamma_{j+1} sum_k |w_ik| |x_kj|."""
    Wr = W[rows]
    R = np.abs(Wr).max(axis=1)[:, None]
    C = np.abs(X).max(axis=0)[None, :]
    K = np.arange(1, X.shape[1] + 1)[None, :]
    emu = 2.0 ** -57 * K * R * C
    g = K * U / (1 - K * U)
    fma = g * (np.abs(Wr) @ np.abs(X))
    return emu, fma


@pytest.mark.parametrize("m,n,graded", [(1000, 17, False), (777, 64, False), (1500, 100, True), (700, 130, False),
                                        (513, 256, True), (300, 300, False), (260, 512, False), (129, 65, True)])
def test_emulated_product_within_bound(env, m, n, graded):
    W, X = _operands(m, n, seed=m + n, graded=graded)
    rows = np.arange(m) if m * n <= 200_000 else np.random.default_rng(1).choice(m, 200_000 // n, replace=False)
    exact = O.product_rounded(W, X, rows=rows)
    emu_b, fma_b = _bounds(W, X, rows)
    Qe = _run(env, W, X, 0)[rows]
    Qf = _run(env, W, X, 1)[rows]
    err_e = np.abs(Qe - exact)
    err_f = np.abs(Qf - exact)
    assert np.all(err_e <= 2 * U * np.abs(exact) + emu_b), float(np.max(err_e / (2 * U * np.abs(exact) + emu_b)))
    assert np.all(err_f <= U * np.abs(exact) + fma_b + 1e-300)
    if not graded:   # FP64 quality on columns of one scale (the case of W = A R_s^{-1})
        assert np.linalg.norm(err_e) <= 2.0 * np.linalg.norm(err_f) + 1e-300


def test_emulated_product_full_height_sampled_rows(env):
    m, n = 1 << 20, 128
    W, X = _operands(m, n, seed=5)
    rows = np.random.default_rng(2).choice(m, 1500, replace=False)
    rows = np.concatenate([rows, [0, 127, 128, m - 1]])
    exact = O.product_rounded(W, X, rows=rows)
    emu_b, _ = _bounds(W, X, rows)
    Qe = _run(env, W, X, 0)[rows]
    assert np.all(np.abs(Qe - exact) <= 2 * U * np.abs(exact) + emu_b)


def test_emulated_product_edge_cases(env):
    torch, M = env
    m, n = 300, 70
    W, X = _operands(m, n, seed=9)
    W[3] = 0.0                                   # zero row
    W[4] = -0.0
    W[5, 10] = 2.0 ** -1070                      # subnormal entry: sliced to zero against its row
    W[6, :] = 2.0 ** -1000                       # tiny row
    W[7, :] = 2.0 ** 900 * np.sign(W[7, :])      # huge row
    X[:, 20] = 0.0                               # zero column
    exact = O.product_rounded(W, X)
    Qe = _run(env, W, X, 0)
    emu_b, _ = _bounds(W, X, np.arange(m))
    assert np.all(np.abs(Qe - exact) <= 2 * U * np.abs(exact) + emu_b)
    assert np.all(Qe[3] == 0.0) and np.all(Qe[:, 20] == 0.0)
    # a non-finite entry turns its row into NaN; the other rows are unaffected
    W2 = W.copy()
    W2[11, 30] = np.nan
    Q2 = _run(env, W2, X, 0)
    assert np.all(np.isnan(Q2[11]))
    keep = np.arange(m) != 11
    np.testing.assert_array_equal(Q2[keep], Qe[keep])


def test_emulated_product_deterministic(env):
    W, X = _operands(2000, 200, seed=3)
    a = _run(env, W, X, 0)
    b = _run(env, W, X, 0)
    np.testing.assert_array_equal(a, b)


def test_finalize_rejects_bad_arguments(env):
    torch, M = env
    from paper_2606_18411_gb300 import _lib
    lib = _lib.load()
    W = M.empty_colmajor(100, 10)
    X = M.empty_colmajor(10, 10)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.mrcqr_finalize_q(100, 10, W.data_ptr(), 99, X.data_ptr(), 10, 0, s) == 1
    assert lib.mrcqr_finalize_q(100, 10, W.data_ptr(), 100, X.data_ptr(), 10, 2, s) == 1
    assert lib.mrcqr_finalize_q(100, 513, W.data_ptr(), 100, X.data_ptr(), 513, 0, s) == 1
    assert lib.mrcqr_finalize_q(100, 10, W.data_ptr(), 100, W.data_ptr(), 10, 0, s) == 1


@pytest.mark.parametrize("prec", ["fp16", "fp32", "fp64"])
@pytest.mark.parametrize("m,n,kappa", [(30000, 128, 1e4), (20000, 200, 1e10), (9000, 33, 1e15)])
def test_factorization_with_emulated_products(env, prec, m, n, kappa):
    torch, M = env
    A = inputs.make_matrix(m, n, kappa, seed=n)
    Ad = M.to_colmajor(A)
    res = {}
    for fp in (0, 1):
        Q = M.empty_colmajor(m, n)
        R = M.empty_colmajor(n, n)
        M.factor_ex(Ad, Q, R, prec=prec, seed=4, fp64_products=fp)
        st = M.last_status()
        assert st["status"] == "OK", (fp, st)
        Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
        res[fp] = O.orthogonality_error(Qh)[0], O.residual_error(A, Qh, Rh)[0]
        assert res[fp][0] <= 1e-13 and res[fp][1] <= 1e-13, (fp, res[fp])
    # same R (the product only changes Q) and comparable orthogonality
    assert res[0][0] <= 3.0 * res[1][0] + 2e-15


def _gram_operand(m, n, seed, graded=False):
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((m, n)) / np.sqrt(m)
    if graded:
        W *= 2.0 ** rng.integers(-12, 12, (1, n))
        W *= 2.0 ** rng.integers(-6, 6, (m, 1))
    return W


def _gram_check(env, W, cols=None, fro_vs_fma=True):
    torch, M = env
    m, n = W.shape
    cols = np.arange(n) if cols is None else np.asarray(cols)
    Wd = M.to_colmajor(W)
    Ge = M.gram(Wd, fp64_products=0).cpu().numpy()
    Gf = M.gram(Wd, fp64_products=1).cpu().numpy()
    exact = O.product_rounded(np.ascontiguousarray(W[:, cols].T), W)       # rows: cols, all j
    C = np.abs(W).max(axis=0)
    bound = 2 * U * np.abs(exact) + 2.0 ** -57 * m * C[cols][:, None] * C[None, :]
    upper = cols[:, None] <= np.arange(n)[None, :]
    err_e = np.where(upper, np.abs(Ge[cols] - exact), 0.0)
    assert np.all(err_e <= bound), float(np.max(err_e / bound))
    assert np.all(np.tril(Ge, -1) == 0.0)
    if fro_vs_fma:
        err_f = np.where(upper, np.abs(Gf[cols] - exact), 0.0)
        assert np.linalg.norm(err_e) <= 2.0 * np.linalg.norm(err_f) + 1e-300
    return Ge


@pytest.mark.parametrize("m,n,graded", [(1000, 17, False), (5000, 64, False), (3001, 100, True), (2000, 128, False),
                                        (1500, 200, True), (999, 333, False), (255, 40, False), (1, 5, False)])
def test_emulated_gram_within_bound(env, m, n, graded):
    W = _gram_operand(m, n, seed=m * 7 + n, graded=graded)
    _gram_check(env, W, fro_vs_fma=not graded and m > 1)


def test_emulated_gram_max_width_sampled(env):
    W = _gram_operand(700, 512, seed=21)
    cols = np.array([0, 63, 64, 127, 128, 255, 256, 300, 383, 384, 447, 448, 511])
    _gram_check(env, W, cols=cols)


def test_emulated_gram_full_height_sampled(env):
    m, n = 1 << 20, 128
    W = _gram_operand(m, n, seed=22)
    _gram_check(env, W, cols=[77], fro_vs_fma=False)


def test_emulated_gram_edge_cases(env):
    torch, M = env
    W = _gram_operand(3000, 70, seed=23)
    W[:, 5] = 0.0                       # zero column
    W[100, 9] = 1e3                     # one spike dominating its column's reference exponent
    Ge = _gram_check(env, W, fro_vs_fma=False)
    assert np.all(Ge[:, 5] == 0.0) and np.all(Ge[5, :] == 0.0)
    W2 = W.copy()
    W2[17, 30] = np.inf
    G2 = M.gram(M.to_colmajor(W2)).cpu().numpy()
    bad = np.zeros_like(G2, dtype=bool)
    bad[30, 30:] = True
    bad[:31, 30] = True
    assert np.all(np.isnan(G2[bad]))
    good = np.triu(~bad)
    np.testing.assert_array_equal(G2[good], Ge[good])


def test_emulated_gram_deterministic_and_symmetric_in_rows(env):
    torch, M = env
    W = _gram_operand(40000, 96, seed=24)
    perm = np.random.default_rng(0).permutation(40000)
    a = M.gram(M.to_colmajor(W)).cpu().numpy()
    b = M.gram(M.to_colmajor(W[perm])).cpu().numpy()   # a row permutation changes every slab's content
    np.testing.assert_array_equal(a, b)


# --- FP64 sketch as an emulated GEMM --------------------------------------
def _sketch_exact(A, idx, d, s):
    """Correctly rounded sum_j F_kj d_j A_jc per sampled row (F the orthonormal
    DCT row without its sqrt(2/m) c_k factor), times sqrt(2/s) c_k."""
    m = A.shape[0]
    F = np.stack([O.dct_row(int(k), m) / O.dct_coefficient(int(k), m) for k in idx])   # cos values
    P = O.product_rounded(F, d[:, None] * A)
    coef = np.sqrt(2.0 / s) * np.where(idx == 0, np.sqrt(0.5), 1.0)
    return coef[:, None] * P, coef, F


@pytest.mark.parametrize("variant", [3, 5])
@pytest.mark.parametrize("m,n,s", [(3000, 40, 80), (4097, 33, 66), (700, 130, 260), (257, 5, 10)])
def test_emulated_sketch_against_exact(env, m, n, s, variant):
    # 3: digits sliced per work item; 5: digit planes of D A and the table's digits
    torch, M = env
    A = inputs.make_matrix(m, n, 1e12, seed=m + n)
    Y = M.sketch(M.to_colmajor(A), s, "fp64", seed=3, variant=variant).cpu().numpy()
    assert M.last_sketch_variant() == variant
    d, idx = O.rademacher(m, 3), O.sample_rows(m, s, 3)
    ref, coef, F = _sketch_exact(A, idx, d, s)
    # the table's cos values and numpy's may differ by an ulp each: 2^-52 sum |A|
    C = np.abs(A).max(axis=0)[None, :]
    bound = coef[:, None] * (2.0 ** -52 * np.abs(A).sum(axis=0)[None, :] + 2.0 ** -57 * m * C) + 2 * U * np.abs(ref)
    err = np.abs(Y - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("m,n,s", [(1 << 16, 128, 256), (20000, 200, 400), (30001, 64, 192), (5000, 512, 1024)])
def test_emulated_sketch_matches_fma_sketch(env, m, n, s):
    torch, M = env
    A = inputs.make_matrix(m, n, 1e14, seed=7 + n)
    Ad = M.to_colmajor(A)
    Ye = M.sketch(Ad, s, "fp64", seed=9).cpu().numpy()
    Yf = M.sketch(Ad, s, "fp64", seed=9, variant=1).cpu().numpy()
    ref = O.sketch(A, O.sample_rows(m, s, 9), O.rademacher(m, 9)) if m * s <= 1 << 24 else Yf
    # both references carry FP64 summation error (~u sqrt(m) relative); the emulated sum has none
    assert np.linalg.norm(Ye - ref) <= 5e-14 * np.linalg.norm(ref)
    assert np.linalg.norm(Ye - Yf) <= 5e-14 * np.linalg.norm(Yf)


def test_emulated_sketch_odd_ld_and_nonfinite(env):
    torch, M = env
    m, n = 5000, 30
    A = inputs.make_matrix(m, n, 1e4, seed=31)
    Y0 = M.sketch(M.to_colmajor(A), 2 * n, "fp64", seed=1).cpu().numpy()
    Y1 = M.sketch(M.to_colmajor(A, ld=m + 1), 2 * n, "fp64", seed=1).cpu().numpy()   # no alignment needed
    assert M.last_sketch_variant() == 5
    np.testing.assert_array_equal(Y0, Y1)
    Y3 = M.sketch(M.to_colmajor(A, ld=m + 1), 2 * n, "fp64", seed=1, variant=3).cpu().numpy()
    assert M.last_sketch_variant() == 3
    np.testing.assert_array_equal(Y0, Y3)
    A[123, 7] = np.nan
    Q = M.empty_colmajor(m, n)
    R = M.empty_colmajor(n, n)
    M.factor_ex(M.to_colmajor(A), Q, R, prec="fp64", seed=1)
    assert M.last_status()["status"] == "NONFINITE"


def test_factorization_fp64_sketch_emulated_vs_fma(env):
    torch, M = env
    m, n = 40000, 96
    A = inputs.make_matrix(m, n, 1e16, seed=77)
    Ad = M.to_colmajor(A)
    out = []
    for fp in (0, 1):
        Q = M.empty_colmajor(m, n)
        R = M.empty_colmajor(n, n)
        M.factor_ex(Ad, Q, R, prec="fp64", seed=2, escalate=False, fp64_products=fp)
        st = M.last_status()
        assert st["status"] == "OK" and st["prec_used"] == "fp64"
        Qh, Rh = Q.cpu().numpy(), R.cpu().numpy()
        out.append((O.orthogonality_error(Qh)[0], O.residual_error(A, Qh, Rh)[0]))
    for o, r in out:
        assert o <= 1e-13 and r <= 1e-13


# --- W = A R^{-1} with emulated off-diagonal updates ------------------------
def _upper(n, kind, seed):
    rng = np.random.default_rng(seed)
    R = np.triu(rng.standard_normal((n, n)) * 0.3) + np.diag(1.0 + rng.random(n))
    if kind == "graded":                       # diagonal from 1 down to 1e-10, rows scaled with it
        R = np.diag(10.0 ** (-10.0 * np.arange(n) / max(n - 1, 1))) @ R
    elif kind == "cliff":                      # second half of the rows 1e-12 smaller
        R[n // 2:] *= 1e-12
    return R


@pytest.mark.parametrize("m,n,kind", [(1000, 17, "plain"), (777, 64, "graded"), (1500, 100, "cliff"),
                                      (700, 130, "plain"), (513, 256, "graded"), (300, 512, "plain"),
                                      (129, 33, "cliff"), (5000, 16, "plain")])
def test_emulated_trsm_backward_error(env, m, n, kind):
    torch, M = env
    rng = np.random.default_rng(m * 3 + n)
    A = rng.standard_normal((m, n))
    R = _upper(n, kind, seed=n)
    Ad, Rd = M.to_colmajor(A), M.to_colmajor(R)
    We = M.trsm(Ad, Rd, fp64_products=0).cpu().numpy()
    Wf = M.trsm(Ad, Rd, fp64_products=1).cpu().numpy()
    rows = np.arange(m) if m * n <= 100_000 else rng.choice(m, 100_000 // n, replace=False)
    scale = np.linalg.norm(np.abs(We[rows]) @ np.abs(R))
    res = {}
    for name, Wx in (("emu", We), ("fma", Wf)):
        WR = O.product_rounded(Wx[rows], R)
        res[name] = np.linalg.norm(A[rows] - WR)
    # backward stable like substitution: ||A - W R|| = O(n u) || |W| |R| ||
    assert res["emu"] <= 4 * n * U * scale, (res, scale)
    assert res["emu"] <= 4 * res["fma"] + 8 * U * scale, res
    if n <= 64 and kind == "plain":   # well-conditioned triangle: the oracle's substitution agrees closely
        Wo = O.trsm_right_upper(A[rows], R)
        assert np.linalg.norm(We[rows] - Wo) <= 1e-12 * np.linalg.norm(Wo)


def test_emulated_trsm_full_height_and_ld(env):
    torch, M = env
    m, n = (1 << 20) + 77, 128
    rng = np.random.default_rng(5)
    R = _upper(n, "graded", seed=5)
    At = torch.randn(n, m, dtype=torch.float64, device="cuda").t()           # column-major
    W = M.trsm(At, M.to_colmajor(R)).cpu().numpy()
    rows = np.concatenate([rng.choice(m, 400, replace=False), [0, 127, 128, m - 1]])
    A = At[rows].cpu().numpy()
    WR = O.product_rounded(W[rows], R)
    assert np.linalg.norm(A - WR) <= 4 * n * U * np.linalg.norm(np.abs(W[rows]) @ np.abs(R))
    # odd leading dimensions give the same W
    A2 = M.to_colmajor(A, ld=len(rows) + 3)
    W2 = M.trsm(A2, M.to_colmajor(R, ld=n + 1)).cpu().numpy()
    np.testing.assert_array_equal(W2, M.trsm(M.to_colmajor(A), M.to_colmajor(R)).cpu().numpy())


# The sketch from digit planes forms the same digits as the per-item kernel and sums the same exact
# integers, so Y is bit for bit the same, whatever the transform, the leading dimension or the shape.
@pytest.mark.parametrize("m,n,s,ld,transform", [(1 << 16, 128, 256, 0, "dct"), (20000, 200, 400, 20001, "dct"),
                                                 (5000, 512, 1024, 0, "dct"), (4099, 1, 2, 4100, "dct"),
                                                 (33333, 70, 210, 0, "rfft"), (12288, 64, 128, 12289, "rfft_reim")])
def test_planes_sketch_bit_exact(env, m, n, s, ld, transform):
    torch, M = env
    A = inputs.make_matrix(m, n, 1e14, seed=100 + n)
    Ad = M.to_colmajor(A, ld=ld or None)
    if transform == "dct":
        Yp = M.sketch(Ad, s, "fp64", seed=21, variant=5).cpu().numpy()
        assert M.last_sketch_variant() == 5
        Yi = M.sketch(Ad, s, "fp64", seed=21, variant=3).cpu().numpy()
        assert M.last_sketch_variant() == 3
    else:
        c = s // 2 if transform == "rfft_reim" else s
        Yp = M.sketch_transform(Ad, c, transform, prec="fp64", seed=21, variant=5).cpu().numpy()
        assert M.last_sketch_variant() == 5
        Yi = M.sketch_transform(Ad, c, transform, prec="fp64", seed=21, variant=3).cpu().numpy()
        assert M.last_sketch_variant() == 3
    np.testing.assert_array_equal(Yp, Yi)


# A factorization writes the planes into its Q buffer in row chunks of at most half of Q: 2 chunks at
# m = 2^16 with ldq = m, 3 at m = 2^16 + 1, 1 with a Q buffer of more than twice the rows; below 2048 rows the
# per-item kernel runs.  Q and R are bit for bit those of the per-item sketch.
@pytest.mark.parametrize("m,n,ldq,planes", [(1 << 16, 64, 0, True), ((1 << 16) + 1, 48, 0, True),
                                             (9000, 100, 20000, True), (1500, 16, 0, False)])
def test_factor_planes_sketch_uses_q_buffer(env, m, n, ldq, planes):
    torch, M = env
    A = inputs.make_matrix(m, n, 1e14, seed=300 + n)
    Ad = M.to_colmajor(A)
    outs = []
    for variant in (0, 3):
        Q = M.empty_colmajor(m, n, ld=ldq or None)
        R = M.empty_colmajor(n, n)
        M.factor_ex(Ad, Q, R, prec="fp64", seed=4, escalate=False, sketch_variant=variant)
        st = M.last_status()
        assert st["status"] == "OK" and st["ortho_fro"] <= 1e-13, st
        assert M.last_sketch_variant() == (5 if (variant == 0 and planes) else 3)
        outs.append((Q[:m].cpu().numpy(), R.cpu().numpy()))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
