"""Plain CPU oracle of MRCQR (Algorithm 2 of "Numerically Stable Cholesky-QR on
GPU via Mixed-Precision Randomized Preconditioning", Garrison, Chen, Ipsen).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` use it.  It shares no code, tables or constants with the
CUDA path: every step is written out again here from its definition, slowly
and in FP64 (numpy), so that it can be read against the paper.

Steps, in the paper's order and notation:

* Algorithm 2 step 1 (Sec. II-A): Rademacher signs D and c sampled row indices
  S.  The paper leaves the random generator open; here both come from
  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from that
  paper's round function and constants:
    d_i = 1 - 2 * (Philox(key=seed, ctr=(i, 0, 0, 0)).word0 & 1)
    S   = Floyd's sampling of c distinct values of {0..m-1}, the draw for
          j in [m-c, m) being r = (Philox(key=seed, ctr=(j, 1, 0, 0)).word0
          * (j + 1)) >> 32, sorted ascending.
* Algorithm 2 steps 2-4 (DiagMult, transform, Select; Sec. II-A): the sketch
  Y = sqrt(m/c) * P F D A with F the orthonormal DCT-II
    F_kj = sqrt(2/m) * c_k * cos(pi * k * (2j + 1) / (2m)),
    c_0 = 1/sqrt(2), c_k = 1 otherwise,
  built here as an explicit dense matrix, row by row, with the phase reduced
  exactly as an integer r = k (2j + 1) mod 4m.  The paper's own transform,
  the real part of a column-wise real FFT over c of the floor(m/2) + 1 bins
  with scale sqrt(c/m) (and the variant that also keeps the imaginary parts),
  is here too (``rfft_sketch``, ``sample_bins``); the orthonormal DCT-II with
  scale sqrt(m/c) is the library's default.  A scalar scale of the sketch
  cancels in R_s^{-1} ... R, see ``mrcqr``.
* Algorithm 2 step 5 (SketchQR): Householder QR of Y, normalised to
  diag(R_s) > 0.
* Algorithm 2 steps 6-8 (Stage 2, Algorithm 1 on A R_s^{-1}, Sec. II-A):
  W = A R_s^{-1} by substitution, G = W^T W, Cholesky G = R_c^T R_c,
  Q = W R_c^{-1} by substitution.
* Algorithm 2 step 9: R = R_c R_s.
* Checks (Eq. 1, Fig. 1): ||I - Q^T Q|| and ||A - QR|| / ||A|| with the sums
  in double-double (``ddcheck.c``), Theorem 1's bound and the CholQR probe
  bound (Sec. II-C).

Reduced-precision sketches (Sec. II-B) are emulated by rounding the
sign-flipped input and the transform entries to the sketch precision's
significand before an FP64 product: an error model of fl_p, used only to
separate rounding error from defects.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular as scipy_solve_triangular

U_FP64 = 2.0 ** -53
# unit roundoff of the sketch precisions (round to nearest)
UNIT_ROUNDOFF = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8, "fp32": 2.0 ** -24, "fp64": 2.0 ** -53}
SIGNIFICAND_BITS = {"fp16": 11, "bf16": 8, "fp32": 24, "fp64": 53}
PRECISIONS = ("fp16", "bf16", "fp32", "fp64")

# ---------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11, Sec. 4 "Philox"): 10 rounds of the
# 4x32 round function with multipliers M0, M1 and Weyl key increments W0, W1.
_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 of counter (c0, c1, c2, c3) under key (k0, k1).

    Inputs are scalars or uint arrays (broadcast); returns four uint32 arrays.
    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 as 64-bit
    products, then c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is
    bumped by (W0, W1) between rounds."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(k0) & _MASK32
    k1 = int(k1) & _MASK32
    m0 = np.uint64(_M0)
    m1 = np.uint64(_M1)
    sh = np.uint64(32)
    msk = np.uint64(_MASK32)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> sh, p0 & msk
        hi1, lo1 = p1 >> sh, p1 & msk
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return (c0.astype(np.uint32), c1.astype(np.uint32), c2.astype(np.uint32), c3.astype(np.uint32))


def seed_key(seed: int):
    """The 64-bit sketch seed as the Philox key (low word, high word)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & _MASK32, seed >> 32


def rademacher(m: int, seed: int) -> np.ndarray:
    """Diagonal of D (Algorithm 2 step 1): d_i in {+1, -1}, i < m."""
    k0, k1 = seed_key(seed)
    w0, _, _, _ = philox4x32_10(np.arange(m, dtype=np.uint64), 0, 0, 0, k0, k1)
    return 1.0 - 2.0 * (w0 & 1).astype(np.float64)


def sample_rows(m: int, s: int, seed: int) -> np.ndarray:
    """The sample set S (Algorithm 2 step 1): s distinct row indices of the
    transformed matrix, uniform without replacement (Floyd's algorithm),
    sorted ascending.  Pure-Python loop: s is at most a few thousand."""
    if not (0 < s <= m):
        raise ValueError("need 0 < s <= m")
    k0, k1 = seed_key(seed)
    js = np.arange(m - s, m, dtype=np.uint64)
    u, _, _, _ = philox4x32_10(js, 1, 0, 0, k0, k1)
    chosen = set()
    for j, uj in zip(js.tolist(), u.tolist()):
        r = (uj * (j + 1)) >> 32          # uniform on {0, ..., j}
        chosen.add(j if r in chosen else r)
    return np.array(sorted(chosen), dtype=np.int64)


# ---------------------------------------------------------------------------
# Orthonormal DCT-II and the dense sketch operator (Algorithm 2 steps 2-4)

def dct_coefficient(k: int, m: int) -> float:
    return math.sqrt(2.0 / m) * (1.0 / math.sqrt(2.0) if k == 0 else 1.0)


def dct_row(k: int, m: int) -> np.ndarray:
    """Row k of the orthonormal DCT-II matrix F (length m)."""
    j = np.arange(m, dtype=np.int64)
    r = (np.int64(k) * (2 * j + 1)) % (4 * m)           # exact integer phase
    return dct_coefficient(k, m) * np.cos(np.pi * r.astype(np.float64) / (2.0 * m))


def dct_matrix(m: int) -> np.ndarray:
    return np.stack([dct_row(k, m) for k in range(m)])


def sketch_row(k: int, m: int, s: int, signs: np.ndarray) -> np.ndarray:
    """One row of S = sqrt(m/s) P F D: sqrt(m/s) * F[k, :] * d."""
    return math.sqrt(m / s) * dct_row(k, m) * signs


def sketch(A: np.ndarray, idx: np.ndarray, signs: np.ndarray, rows_per_block: int = 16) -> np.ndarray:
    """Y = S A in FP64.  S is built explicitly row by row; each block of rows
    is applied with one matrix product."""
    m, n = A.shape
    s = len(idx)
    Y = np.empty((s, n))
    for b in range(0, s, rows_per_block):
        ks = idx[b:b + rows_per_block]
        Sb = np.stack([sketch_row(int(k), m, s, signs) for k in ks])
        Y[b:b + len(ks)] = Sb @ A
    return Y


def round_significand(x: np.ndarray, bits: int) -> np.ndarray:
    """Round FP64 values to ``bits`` significand bits, round-to-nearest-even,
    directly from the FP64 bit pattern (no intermediate rounding).  The
    exponent range of the target format is not modelled: callers scale the
    values into its normal range first."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if bits >= 53:
        return x.copy()
    drop = np.uint64(53 - bits)
    b = x.view(np.uint64)
    one = np.uint64(1)
    half = one << (drop - one)
    lsb = (b >> drop) & one
    r = ((b + (half - one) + lsb) >> drop) << drop
    out = r.view(np.float64).copy()
    out[~np.isfinite(x)] = x[~np.isfinite(x)]
    out[x == 0] = x[x == 0]
    return out


def column_scale_exponents(A: np.ndarray, target_exp: int = 13) -> np.ndarray:
    """Per-column power-of-two exponents e_j with max_i |a_ij| 2^e_j in
    [2^target_exp, 2^(target_exp+1)); zero columns get e_j = 0.  (Keeps the
    FP16 sketch clear of underflow, the breakdown mode named in Fig. 1.)"""
    amax = np.max(np.abs(A), axis=0)
    e = np.zeros(A.shape[1], dtype=np.int64)
    nz = amax > 0
    _, ex = np.frexp(amax[nz])               # amax = f * 2^ex, f in [0.5, 1)
    e[nz] = target_exp + 1 - ex
    return e


def sketch_emulated(A: np.ndarray, idx: np.ndarray, signs: np.ndarray, prec: str) -> np.ndarray:
    """Error model of the precision-p sketch: fl_p(D A 2^e) and fl_p(S entries),
    products and sums exact-ish in FP64, then the scale 2^-e undone."""
    bits = SIGNIFICAND_BITS[prec]
    m, n = A.shape
    s = len(idx)
    e = column_scale_exponents(A)
    X = round_significand(signs[:, None] * np.ldexp(A, e[None, :]), bits).reshape(m, n)
    c = math.sqrt(m / s)
    Y = np.empty((s, n))
    for i, k in enumerate(idx):
        row = round_significand(dct_row(int(k), m), bits)
        Y[i] = c * (row @ X)
    return np.ldexp(Y, -e[None, :])


# ---------------------------------------------------------------------------
# The paper's own transform (Algorithm 2 as printed, Sec. II-A): the real FFT
# of each sign-flipped column, c of its floor(m/2) + 1 distinct bins (a real
# column's spectrum is Hermitian), the real parts scaled by sqrt(c/m); the
# variant of Sec. II-A that keeps the imaginary parts as well stacks them
# below, a 2c x n sketch.  Bins are 0-based here (the paper's bin k + 1).

TRANSFORMS = ("dct", "rfft", "rfft_reim")


def sample_bins(m: int, c: int, seed: int) -> np.ndarray:
    """The sampled bins of the real-FFT sketch (Algorithm 2 step 1): c
    distinct values of {0..floor(m/2)}, uniform without replacement, by the
    Floyd draw of ``sample_rows`` over that population, sorted ascending."""
    return sample_rows(m // 2 + 1, c, seed)


def dft_phase(k: int, m: int) -> np.ndarray:
    """k j mod m for j < m, exact in integers: row k of the DFT is
    exp(-2 pi i (k j mod m) / m)."""
    j = np.arange(m, dtype=np.int64)
    return (np.int64(k) * j) % m


def rfft_re_row(k: int, m: int) -> np.ndarray:
    """Real part of row k of the unnormalised DFT: cos(2 pi k j / m)."""
    return np.cos(2.0 * np.pi * dft_phase(k, m).astype(np.float64) / m)


def rfft_im_row(k: int, m: int) -> np.ndarray:
    """Imaginary part of row k of the unnormalised DFT: -sin(2 pi k j / m)."""
    return -np.sin(2.0 * np.pi * dft_phase(k, m).astype(np.float64) / m)


def rfft_rows(bins: np.ndarray, imag: bool = False):
    """The sketch's rows in order: (part, bin) for the Re rows of the bins,
    then, with ``imag``, their Im rows."""
    rows = [("re", int(k)) for k in bins]
    if imag:
        rows += [("im", int(k)) for k in bins]
    return rows


def rfft_sketch_row(part: str, k: int, m: int, c: int, signs: np.ndarray) -> np.ndarray:
    """One row of S = sqrt(c/m) P [Re F; Im F] D (F the unnormalised DFT)."""
    row = rfft_re_row(k, m) if part == "re" else rfft_im_row(k, m)
    return math.sqrt(c / m) * row * signs


def rfft_sketch(A: np.ndarray, bins: np.ndarray, signs: np.ndarray, imag: bool = False,
                rows_per_block: int = 16) -> np.ndarray:
    """Y = S A in FP64 (Algorithm 2 steps 2-4 with the real FFT), S built
    explicitly row by row as ``sketch`` does for the DCT."""
    m, n = A.shape
    c = len(bins)
    rows = rfft_rows(bins, imag)
    Y = np.empty((len(rows), n))
    for b in range(0, len(rows), rows_per_block):
        blk = rows[b:b + rows_per_block]
        Sb = np.stack([rfft_sketch_row(part, k, m, c, signs) for part, k in blk])
        Y[b:b + len(blk)] = Sb @ A
    return Y


def rfft_sketch_emulated(A: np.ndarray, bins: np.ndarray, signs: np.ndarray, prec: str,
                         imag: bool = False) -> np.ndarray:
    """Error model of the precision-p real-FFT sketch, as ``sketch_emulated``:
    fl_p(D A 2^e) and fl_p(cos / sin entries), products in FP64, the scale
    sqrt(c/m) 2^-e applied last."""
    bits = SIGNIFICAND_BITS[prec]
    m, n = A.shape
    c = len(bins)
    e = column_scale_exponents(A)
    X = round_significand(signs[:, None] * np.ldexp(A, e[None, :]), bits).reshape(m, n)
    rows = rfft_rows(bins, imag)
    Y = np.empty((len(rows), n))
    for i, (part, k) in enumerate(rows):
        row = round_significand(rfft_re_row(k, m) if part == "re" else rfft_im_row(k, m), bits)
        Y[i] = row @ X
    return np.ldexp(Y * math.sqrt(c / m), -e[None, :])


# ---------------------------------------------------------------------------
# Small dense factorizations (Algorithm 1 and Algorithm 2 steps 5-9)

def householder_qr(Y: np.ndarray, want_q: bool = False, dtype=np.float64):
    """Thin QR of Y (c x n, c >= n) by Householder reflections, R normalised
    to a positive diagonal (rows of R, columns of Q flipped)."""
    R = np.array(Y, dtype=dtype, copy=True)
    c, n = R.shape
    vs = []
    for j in range(n):
        x = R[j:, j].copy()
        normx = np.sqrt(np.dot(x, x))
        v = x
        if normx == 0:
            vs.append(None)
            continue
        alpha = -normx if x[0] >= 0 else normx
        v[0] = x[0] - alpha
        vnorm = np.sqrt(np.dot(v, v))
        if vnorm == 0:
            vs.append(None)
            continue
        v = v / vnorm
        R[j:, j:] -= dtype(2) * np.outer(v, v @ R[j:, j:])
        vs.append(v)
    Rn = np.triu(R[:n, :]).astype(np.float64)
    sgn = np.where(np.diag(Rn) < 0, -1.0, 1.0)
    Rn = Rn * sgn[:, None]
    if not want_q:
        return Rn
    Q = np.zeros((c, n))
    Q[:n, :n] = np.eye(n)
    for j in reversed(range(n)):
        v = vs[j]
        if v is None:
            continue
        v = v.astype(np.float64)
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    return Q * sgn[None, :], Rn


def trsm_right_upper(A: np.ndarray, R: np.ndarray) -> np.ndarray:
    """W with W R = A (R upper triangular) by substitution: for each row a of
    A, w_j = (a_j - sum_{k<j} w_k R_kj) / R_jj, all rows at once."""
    m, n = A.shape
    W = np.empty((m, n))
    for j in range(n):
        acc = A[:, j] - W[:, :j] @ R[:j, j] if j else A[:, j].copy()
        W[:, j] = acc / R[j, j]
    return W


def two_product(a: np.ndarray, b: np.ndarray):
    """Error-free product a * b = p + e (Dekker 1971, with Veltkamp's split
    into 26-bit halves); exact unless a product under- or overflows."""
    def split(x):
        c = 134217729.0 * x          # 2^27 + 1
        hi = c - (c - x)
        return hi, x - hi
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def product_rounded(W: np.ndarray, X: np.ndarray, rows=None) -> np.ndarray:
    """W X with every entry the exact sum sum_k W_ik X_kj rounded once to FP64
    (the reference for the Q = W R_c^{-1} product of Algorithm 1 step 3 when
    it is evaluated exactly or in emulated FP64): each product split into
    p + e by ``two_product``, the 2K terms summed by math.fsum, which returns
    the correctly rounded sum.  ``rows`` restricts the result to those rows."""
    rows = np.arange(W.shape[0]) if rows is None else np.asarray(rows)
    out = np.empty((len(rows), X.shape[1]))
    for t, i in enumerate(rows):
        p, e = two_product(W[i][:, None], X)          # K x n
        for j in range(X.shape[1]):
            out[t, j] = math.fsum(np.concatenate([p[:, j], e[:, j]]).tolist())
    return out


class CholeskyBreakdown(ArithmeticError):
    pass


def cholesky_upper(G: np.ndarray) -> np.ndarray:
    """Upper R with R^T R = G (Algorithm 1 step 2), column by column.
    Raises CholeskyBreakdown on a non-positive or non-finite pivot."""
    n = G.shape[0]
    R = np.zeros((n, n))
    for j in range(n):
        d = G[j, j] - np.dot(R[:j, j], R[:j, j])
        if not (d > 0) or not np.isfinite(d):
            raise CholeskyBreakdown(f"pivot {j}: {d}")
        R[j, j] = math.sqrt(d)
        for i in range(j + 1, n):
            R[j, i] = (G[j, i] - np.dot(R[:j, j], R[:j, i])) / R[j, j]
    return R


def cholqr(A: np.ndarray):
    """Algorithm 1: G = A^T A, G = R^T R, Q = A R^{-1}."""
    G = A.T @ A
    R = cholesky_upper(G)
    Q = trsm_right_upper(A, R)
    return Q, R


def cholqr2(A: np.ndarray):
    """CholQR2 (Sec. I-A, the comparison method of the stability experiment):
    Algorithm 1 run twice, Q1, R1 = CholQR(A); Q, R2 = CholQR(Q1); R = R2 R1.
    Raises CholeskyBreakdown when the first Gram matrix is not numerically
    positive definite (kappa_2(A) beyond about u^{-1/2})."""
    Q1, R1 = cholqr(A)
    Q, R2 = cholqr(Q1)
    return Q, np.triu(R2 @ R1)


@dataclass
class MRCQRResult:
    Q: np.ndarray
    R: np.ndarray
    Rs: np.ndarray
    Rc: np.ndarray
    Y: np.ndarray
    idx: np.ndarray
    signs: np.ndarray
    extra: dict = field(default_factory=dict)


def sketch_rows_for(n: int, s_factor: int = 2) -> int:
    return s_factor * n


def mrcqr(A: np.ndarray, seed: int = 0, prec: str = "fp64", s: int | None = None,
          sketch_scale: float = 1.0, transform: str = "dct") -> MRCQRResult:
    """Algorithm 2 with sketch precision ``prec`` (fp64: the exact FP64 sketch;
    otherwise the fl_p error model of ``sketch_emulated`` and a sketch QR in
    FP32 as the paper does for half precision, Sec. II-A).  ``transform``:
    "dct" (s sampled DCT-II rows), "rfft" (Re of s sampled real-FFT bins) or
    "rfft_reim" (Re and Im of s bins, a 2s x n sketch)."""
    m, n = A.shape
    if s is None:
        s = sketch_rows_for(n)
    signs = rademacher(m, seed)
    if transform == "dct":
        idx = sample_rows(m, s, seed)
        exact = lambda: sketch(A, idx, signs)
        emulated = lambda: sketch_emulated(A, idx, signs, prec)
    elif transform in ("rfft", "rfft_reim"):
        idx = sample_bins(m, s, seed)
        imag = transform == "rfft_reim"
        exact = lambda: rfft_sketch(A, idx, signs, imag)
        emulated = lambda: rfft_sketch_emulated(A, idx, signs, prec, imag)
    else:
        raise ValueError(f"unknown transform {transform!r}")
    if prec == "fp64":
        Y = exact()
        Rs = householder_qr(Y * sketch_scale)
    else:
        Y = emulated()
        Rs = householder_qr((Y * sketch_scale).astype(np.float32), dtype=np.float32)
    W = trsm_right_upper(A, Rs)
    G = W.T @ W
    Rc = cholesky_upper(G)
    Q = trsm_right_upper(W, Rc)
    R = Rc @ Rs
    return MRCQRResult(Q=Q, R=np.triu(R), Rs=Rs, Rc=Rc, Y=Y, idx=idx, signs=signs)


def precision_rule(kappa: float) -> str:
    """Sketch precision from the regime of kappa_2(A) (Sec. II-B/II-C):
    half up to 1e4, single up to 1e8, double above (boundaries inclusive)."""
    if kappa <= 1e4:
        return "fp16"
    if kappa <= 1e8:
        return "fp32"
    return "fp64"


def theorem1_bound(kappa_A1: float, eps: float, kappa_Rs: float) -> float:
    """Theorem 1: kappa(A (R_s + E)^{-1}) <= kappa(A R_s^{-1}) (1 + eps k)/(1 - eps k)
    with eps = ||E||_2 / ||R_s||_2 and k = kappa_2(R_s); needs eps k < 1."""
    t = eps * kappa_Rs
    if t >= 1:
        return math.inf
    return kappa_A1 * (1 + t) / (1 - t)


def probe_kappa_lower(q: float, u: float = U_FP64) -> float:
    """CholQR probe (Sec. II-C): kappa_2(A) >= sqrt(q / (u (1 + q))) with
    q = ||I - Q^T Q||_2 of a CholQR run."""
    return math.sqrt(q / (u * (1.0 + q)))


# ---------------------------------------------------------------------------
# Regime classification without learning (Sec. II-C): the CholQR probe and the
# block 1-norm estimate on A^T A.  Regime 0 = half, 1 = single, 2 = double,
# from an estimate of kappa_2(A) by ``precision_rule``'s thresholds.

REGIME_PRECISIONS = ("fp16", "fp32", "fp64")


def regime_of(kappa: float) -> int:
    """Regime index of a kappa_2 estimate (``precision_rule``; inf -> 2)."""
    return REGIME_PRECISIONS.index(precision_rule(kappa))


def cholqr_probe(A: np.ndarray, u: float = U_FP64):
    """(kappa estimate, q): Algorithm 1 on A, q = ||I - Q^T Q||_2 (sums in
    double-double), and the bound kappa_2(A) >= sqrt(q / (u (1 + q))) of
    Sec. II-C.  A Cholesky breakdown (A^T A not numerically positive
    definite, kappa_2(A) beyond about u^-1/2) gives (inf, inf)."""
    try:
        Q, _ = cholqr(A)
    except CholeskyBreakdown:
        return math.inf, math.inf
    q = orthogonality_error(Q)[0]
    return probe_kappa_lower(q, u), q


def random_sign_column(n: int, seed: int, draw: int) -> np.ndarray:
    """The ``draw``-th random +-1 column of the block 1-norm estimator:
    entry i = 1 - 2 (Philox(key=seed, ctr=(i, 2, draw, 0)).word0 & 1)."""
    k0, k1 = seed_key(seed)
    w0, _, _, _ = philox4x32_10(np.arange(n, dtype=np.uint64), 2, draw, 0, k0, k1)
    return 1.0 - 2.0 * (w0 & 1).astype(np.float64)


def _parallel(x: np.ndarray, y: np.ndarray) -> bool:
    """Two +-1 columns are parallel when they are equal or opposite."""
    return abs(float(x @ y)) == len(x)


def onenorm_estimate(apply_B, apply_Bt, n: int, t: int = 2, itmax: int = 5, seed: int = 0,
                     max_resample: int = 100) -> float:
    """Block 1-norm estimator of Higham and Tisseur (SIAM J. Matrix Anal.
    Appl. 21 (2000), Algorithm 2.4), a lower bound est <= ||B||_1 of a matrix
    seen only through products B X and B^T X (n x t blocks).  Its random +-1
    columns come from ``random_sign_column``; a column parallel to an
    earlier one is redrawn (at most ``max_resample`` times).  For n <= 4 the
    norm is computed exactly from B I (as MATLAB's normest1 does)."""
    if n <= 4:
        return float(np.abs(apply_B(np.eye(n))).sum(axis=0).max())
    draw = 0

    def fresh():
        nonlocal draw
        x = random_sign_column(n, seed, draw)
        draw += 1
        return x

    # starting block: e/n, then random +-1 columns, none parallel to an earlier one
    X = np.empty((n, t))
    X[:, 0] = 1.0
    for j in range(1, t):
        x = fresh()
        for _ in range(max_resample):
            if not any(_parallel(x, X[:, i]) for i in range(j)):
                break
            x = fresh()
        X[:, j] = x
    X /= n
    ind_hist: list[int] = []
    est_old = 0.0
    ind = np.zeros(n, dtype=np.int64)
    S = np.zeros((n, t))
    ind_best = 0
    est = 0.0
    for k in range(1, itmax + 2):
        Y = apply_B(X)
        norms = np.abs(Y).sum(axis=0)
        jbest = int(np.argmax(norms))
        est = float(norms[jbest])
        if est > est_old or k == 2:
            ind_best = int(ind[jbest])
        if k >= 2 and est <= est_old:          # (1) no increase: stop with the previous estimate
            est = est_old
            break
        est_old = est
        S_old = S
        if k > itmax:
            break
        S = np.where(Y >= 0, 1.0, -1.0)
        if all(any(_parallel(S[:, j], S_old[:, i]) for i in range(t)) for j in range(t)):   # (2)
            break
        if t > 1:                              # (3) no column parallel to an earlier one or to S_old
            for j in range(t):
                for _ in range(max_resample):
                    if not (any(_parallel(S[:, j], S[:, i]) for i in range(j)) or
                            any(_parallel(S[:, j], S_old[:, i]) for i in range(t))):
                        break
                    S[:, j] = fresh()
        Z = apply_Bt(S)
        h = np.abs(Z).max(axis=1)
        if k >= 2 and h.max() == h[ind_best]:  # (4)
            break
        order = np.argsort(-h, kind="stable")  # h descending, ties by index
        if t > 1:
            if all(int(i) in ind_hist for i in order[:t]):
                break
            fresh_idx = [int(i) for i in order if int(i) not in ind_hist][:t]
            if len(fresh_idx) < t:
                break
            order = np.array(fresh_idx)
        ind = np.zeros(n, dtype=np.int64)
        X = np.zeros((n, t))
        for j in range(t):
            X[order[j], j] = 1.0
            ind[j] = order[j]
        ind_hist += [int(i) for i in order[:t]]
    return est


def onenorm_regime_estimate(A: np.ndarray, seed: int = 0):
    """(kappa estimate, ||G||_1, est ||G^-1||_1) with G = A^T A: the bound
    kappa_2(A)^2 <= n ||G||_1 ||G^-1||_1 of Sec. II-C, ||G^-1||_1 from the
    block estimator with G^-1 applied through the Cholesky factor
    (G = R^T R: two substitutions).  A Cholesky breakdown gives inf."""
    n = A.shape[1]
    G = A.T @ A
    try:
        R = cholesky_upper(G)
    except CholeskyBreakdown:
        return math.inf, float(np.abs(G).sum(axis=0).max()), math.inf
    solve = lambda X: scipy_solve_triangular(R, scipy_solve_triangular(R, X, trans="T"))
    g1 = float(np.abs(G).sum(axis=0).max())
    est = onenorm_estimate(solve, solve, n, seed=seed)
    return math.sqrt(n * g1 * est), g1, est


def cond2(A: np.ndarray) -> float:
    sv = np.linalg.svd(A, compute_uv=False)
    return float(sv[0] / sv[-1])


# ---------------------------------------------------------------------------
# Double-double checks (compiled C, see ddcheck.c)

_DD = None


def _dd_lib():
    global _DD
    if _DD is None:
        here = os.path.dirname(os.path.abspath(__file__))
        path = os.path.join(here, "libddcheck.so")
        if not os.path.exists(path):
            from . import build as _b
            _b.build_oracle()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        lib.dd_gram_minus_identity.argtypes = [i64, i64, dp, i64, dp]
        lib.dd_gram_minus_identity.restype = None
        lib.dd_residual_columns.argtypes = [i64, i64, dp, i64, dp, i64, dp, i64, dp]
        lib.dd_residual_columns.restype = None
        lib.dd_dot.argtypes = [i64, dp, dp]
        lib.dd_dot.restype = ctypes.c_double
        _DD = lib
    return _DD


def _f64_fortran(X):
    return np.asfortranarray(X, dtype=np.float64)


def _ptr(X):
    return X.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def orthogonality_error(Q: np.ndarray):
    """(||I - Q^T Q||_2, ||I - Q^T Q||_F) with Q^T Q - I summed in
    double-double (Dot2 of Ogita, Rump, Oishi 2005) and rounded once."""
    Q = _f64_fortran(Q)
    m, n = Q.shape
    E = np.zeros((n, n), order="F")
    _dd_lib().dd_gram_minus_identity(m, n, _ptr(Q), m, _ptr(E))
    return float(np.linalg.norm(E, 2)), float(np.linalg.norm(E, "fro")), E


def residual_error(A: np.ndarray, Q: np.ndarray, R: np.ndarray):
    """(||A - QR||_F / ||A||_F, ||A - QR||_2 / ||A||_2) with each entry of
    A - QR accumulated in double-double (R upper triangular)."""
    A = _f64_fortran(A)
    Q = _f64_fortran(Q)
    R = _f64_fortran(np.triu(R))
    m, n = A.shape
    Rres = np.zeros((m, n), order="F")
    _dd_lib().dd_residual_columns(m, n, _ptr(A), m, _ptr(Q), m, _ptr(R), n, _ptr(Rres))
    fro = float(np.linalg.norm(Rres) / np.linalg.norm(A))
    two = float(np.linalg.norm(Rres, 2) / np.linalg.norm(A, 2))
    return fro, two


def dd_dot(x: np.ndarray, y: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(_dd_lib().dd_dot(len(x), _ptr(x), _ptr(y)))
