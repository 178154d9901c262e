"""The seeded input generators that serve both the oracle and the CUDA path:
the spectra of the input recipe (geometric from 1 to 1/kappa, step-cliff,
clustered, log-uniform) and matrices A = U diag(sigma) V^T whose singular
values are those spectra, checked against numpy's SVD (no GPU)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2606_18411_gb300 import inputs


@pytest.mark.parametrize("n", [2, 7, 64])
def test_spectra_definitions(n):
    kappa = 1e8
    g = inputs.spectrum("geometric", n, kappa)
    assert g[0] == 1.0 and abs(g[-1] * kappa - 1.0) < 1e-12
    np.testing.assert_allclose(g[1:] / g[:-1], kappa ** (-1.0 / (n - 1)), rtol=1e-12)
    c = inputs.spectrum("cliff", n, kappa)
    h = (n + 1) // 2
    assert np.all(c[:h] == 1.0) and np.all(c[h:] == 1.0 / kappa)
    k = inputs.spectrum("clustered", n, kappa)
    assert np.all(k[:-1] == 1.0) and k[-1] == 1.0 / kappa
    lu = inputs.spectrum("loguniform", n, kappa, np.random.default_rng(0))
    assert lu[0] == 1.0 and lu[-1] == 1.0 / kappa and np.all(np.diff(lu) <= 0)
    assert np.all((lu >= 1.0 / kappa) & (lu <= 1.0))
    assert np.array_equal(inputs.spectrum("geometric", 1, kappa), np.ones(1))


@pytest.mark.parametrize("kind", inputs.SPECTRA)
@pytest.mark.parametrize("kappa", [1.0, 1e3, 1e6])
def test_make_matrix_has_the_spectrum(kind, kappa):
    m, n = 3000, 24
    A, U, sig, V = inputs.make_matrix(m, n, kappa, kind=kind, seed=17, return_factors=True)
    assert A.flags.f_contiguous
    np.testing.assert_allclose(U.T @ U, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    sv = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(sv, sig, rtol=1e-11 * max(kappa, 1.0), atol=0)
    assert abs(sv[0] / sv[-1] / kappa - 1.0) < 1e-9
    # seeded: the same draw twice, another draw for another seed
    np.testing.assert_array_equal(A, inputs.make_matrix(m, n, kappa, kind=kind, seed=17))
    assert not np.array_equal(A, inputs.make_matrix(m, n, kappa, kind=kind, seed=18))


def test_torch_generator_has_the_spectrum_on_cpu():
    torch = pytest.importorskip("torch")
    m, n, kappa = 5000, 16, 1e5
    A = inputs.make_matrix_torch(m, n, kappa, seed=3, device="cpu", rounds=2)
    assert A.stride(0) == 1   # column-major
    sv = np.linalg.svd(A.numpy(), compute_uv=False)
    np.testing.assert_allclose(sv, inputs.spectrum("geometric", n, kappa), rtol=1e-9)
