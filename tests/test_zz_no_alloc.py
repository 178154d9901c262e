"""The allocation-free sketch QR (mrcqr_sketch_qr_noalloc) agrees with the
allocating entry point (mrcqr_sketch_qr).

The allocation-free call serves callers that cannot allocate device memory
where they need R_s (a foreign memory manager that forbids raw cudaMalloc,
or a loop where an allocation's implicit synchronization is not allowed); it
takes its scratch from one static device array.  Two calls in a row, of
different shapes and precisions, check that the shared scratch carries no
state from one call into the next.  This file is collected last so a failure
here comes after every other test has run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_18411_gb300 import build
    build.build()
    from paper_2606_18411_gb300 import _lib
    from paper_2606_18411_gb300 import mrcqr as M
    return torch, _lib.load(), M


def _noalloc(torch, lib, M, Y, prec):
    s, n = Y.shape
    Rs = M.empty_colmajor(n, n)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.mrcqr_sketch_qr_noalloc(n, s, Y.data_ptr(), M.PREC[prec], Rs.data_ptr(), stream)
    assert rc == 0
    return Rs


def test_noalloc_matches_allocating_sketch_qr_twice(env):
    torch, lib, M = env
    cases = [(64, 128, "fp64", 1), (100, 200, "fp32", 2)]     # two calls in a row, different shapes
    for n, s, prec, seed in cases:
        Yh = inputs.gaussian(s, n, seed=seed) * np.logspace(0, -6, n)[None, :]
        Y = M.to_colmajor(Yh)
        ref = M.sketch_qr(Y, prec).cpu().numpy()
        got = _noalloc(torch, lib, M, Y, prec).cpu().numpy()
        torch.cuda.synchronize()
        tol = 1e-12 if prec == "fp64" else 1e-4
        colerr = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert colerr.max() <= tol, (n, s, prec, colerr.max())
        np.testing.assert_array_equal(np.tril(got, -1), 0)
        assert np.all(np.diag(got) > 0)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, lib, M = env
    stream = torch.cuda.current_stream().cuda_stream
    Y = M.empty_colmajor(600, 129)
    Rs = M.empty_colmajor(129, 129)
    assert lib.mrcqr_sketch_qr_noalloc(129, 600, Y.data_ptr(), 3, Rs.data_ptr(), stream) == 1
    Y2 = M.empty_colmajor(513, 64)
    Rs2 = M.empty_colmajor(64, 64)
    assert lib.mrcqr_sketch_qr_noalloc(64, 513, Y2.data_ptr(), 3, Rs2.data_ptr(), stream) == 1
