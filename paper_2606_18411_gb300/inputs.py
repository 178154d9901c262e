"""Seeded synthetic test matrices (the only module shared by the CUDA path's
tests/bench and the CPU oracle).

It holds no MRCQR arithmetic: it only builds inputs A = U diag(sigma) V^T with
a prescribed 2-norm condition number, the construction of the paper's
stability experiment (Sec. III-B, test-matrix equation), with the spectra used
by the workloads:

* ``geometric``  sigma_i = kappa^(-i/(n-1)), from 1 down to 1/kappa
  (the paper's form kappa^(1/2 - i/(n-1)) is the same up to the scalar
  kappa^(1/2), which changes neither kappa nor the QR factors' shape);
* ``cliff``      half the values 1, the other half 1/kappa;
* ``clustered``  n-1 values equal to 1 and the last one 1/kappa;
* ``loguniform`` sigma_0 = 1, sigma_{n-1} = 1/kappa, the interior drawn
  log-uniformly in [1/kappa, 1] and sorted.

U is the Q factor of an m x n Gaussian matrix and V a Haar-distributed
orthogonal n x n matrix (QR of a Gaussian with the R diagonal made positive).
The paper draws the random matrices uniform on [-1, 1]; the Gaussian draw is
the reading used here (both give orthonormal factors; only sigma fixes kappa).

Every draw comes from ``numpy.random.Generator(Philox(seed))`` so a seed
fixes the matrix on every machine.
"""
from __future__ import annotations

import numpy as np

SPECTRA = ("geometric", "cliff", "clustered", "loguniform")


def spectrum(kind: str, n: int, kappa: float, rng: np.random.Generator | None = None) -> np.ndarray:
    """Singular values (descending, sigma_0 = 1, sigma_{n-1} = 1/kappa)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    if n == 1:
        return np.ones(1)
    lk = np.log(float(kappa))
    if kind == "geometric":
        return np.exp(-lk * np.arange(n) / (n - 1))
    if kind == "cliff":
        h = (n + 1) // 2
        return np.concatenate([np.ones(h), np.full(n - h, 1.0 / kappa)])
    if kind == "clustered":
        return np.concatenate([np.ones(n - 1), [1.0 / kappa]])
    if kind == "loguniform":
        if rng is None:
            raise ValueError("loguniform spectrum needs an rng")
        mid = np.exp(-lk * rng.random(n - 2)) if n > 2 else np.empty(0)
        return np.concatenate([[1.0], np.sort(mid)[::-1], [1.0 / kappa]])
    raise ValueError(f"unknown spectrum {kind!r}")


def _orthonormal_columns(G: np.ndarray) -> np.ndarray:
    q, r = np.linalg.qr(G)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def make_matrix(m: int, n: int, kappa: float, kind: str = "geometric", seed: int = 0,
                return_factors: bool = False):
    """A = U diag(sigma) V^T, m x n FP64, Fortran (column-major) order.

    With ``return_factors`` also returns (U, sigma, V)."""
    if m < n:
        raise ValueError("need m >= n")
    rng = np.random.Generator(np.random.Philox(seed))
    sig = spectrum(kind, n, kappa, rng)
    U = _orthonormal_columns(rng.standard_normal((m, n)))
    V = _orthonormal_columns(rng.standard_normal((n, n)))
    A = np.asfortranarray((U * sig) @ V.T)
    if return_factors:
        return A, U, sig, V
    return A


def orthonormal_matrix(m: int, n: int, seed: int = 0) -> np.ndarray:
    """An m x n matrix with orthonormal columns (kappa = 1), column-major."""
    rng = np.random.Generator(np.random.Philox(seed))
    return np.asfortranarray(_orthonormal_columns(rng.standard_normal((m, n))))


def upper_with_positive_diag(n: int, kappa_scale: float = 1.0, seed: int = 0) -> np.ndarray:
    """A random n x n upper-triangular matrix with positive diagonal; the
    diagonal is graded geometrically from 1 to 1/kappa_scale."""
    rng = np.random.Generator(np.random.Philox(seed))
    R = np.triu(rng.standard_normal((n, n)))
    d = np.exp(-np.log(kappa_scale) * np.arange(n) / max(n - 1, 1))
    R[np.diag_indices(n)] = d
    return R


def gaussian(m: int, n: int, seed: int = 0) -> np.ndarray:
    rng = np.random.Generator(np.random.Philox(seed))
    return np.asfortranarray(rng.standard_normal((m, n)))


def make_matrix_device(m: int, n: int, kappa: float, kind: str = "geometric", seed: int = 0, device="cuda"):
    """Same construction as ``make_matrix`` for large m, on ``device``: U is
    orthonormalised from the seeded Gaussian by two rounds of Gram/Cholesky
    (matrix products on the device, the n x n Cholesky on the host), which
    for a Gaussian m x n (kappa ~ 1) gives orthonormality at the 1e-15 level.
    Input generation only.  Returns a column-major torch float64 tensor."""
    import torch
    rng = np.random.Generator(np.random.Philox(seed))
    sig = spectrum(kind, n, kappa, rng)
    U = torch.from_numpy(rng.standard_normal((n, m))).to(device).t()      # column-major m x n
    for _ in range(2):
        G = (U.t() @ U).cpu().numpy()
        Rinv = np.linalg.inv(np.linalg.cholesky(G).T)
        U = U @ torch.from_numpy(Rinv).to(device)
    V = torch.from_numpy(_orthonormal_columns(rng.standard_normal((n, n)))).to(device)
    B = torch.from_numpy(sig).to(device)[:, None] * V.t()                 # Sigma V^T
    out = torch.empty((n, m), dtype=torch.float64, device=device).t()
    out.copy_(U @ B)
    return out


def make_matrix_torch(m: int, n: int, kappa: float, kind: str = "geometric", seed: int = 0, device="cuda",
                      rounds: int = 1):
    """Like ``make_matrix_device`` but with the Gaussian drawn by torch's
    seeded generator on the device (fast input generation for large batches);
    one Gram/Cholesky round already orthonormalises a Gaussian to ~1e-15.
    Returns a column-major torch float64 tensor."""
    import torch
    rng = np.random.Generator(np.random.Philox(seed))
    sig = spectrum(kind, n, kappa, rng)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    U = torch.randn((n, m), dtype=torch.float64, device=device, generator=g).t()
    for _ in range(rounds):
        G = (U.t() @ U).cpu().numpy()
        Rinv = np.linalg.inv(np.linalg.cholesky(G).T)
        U = U @ torch.from_numpy(Rinv).to(device)
    V = torch.from_numpy(_orthonormal_columns(rng.standard_normal((n, n)))).to(device)
    B = torch.from_numpy(sig).to(device)[:, None] * V.t()
    out = torch.empty((n, m), dtype=torch.float64, device=device).t()
    out.copy_(U @ B)
    return out
