"""The allocation-free sketch QR (mrcqr_sketch_qr_noalloc).

Some callers cannot allocate device memory at the moment they need R_s: code
running under another framework's memory manager that forbids raw
cudaMalloc, or a latency-critical loop where an allocation (and the
synchronization it can bring) is not allowed.  This entry point takes its
scratch from one static device array instead.  The tests check that it

* gives exactly the allocating entry point's R_s (same kernels, no atomics,
  so bit for bit) and the oracle's Householder R_s within the sketch QR's
  tolerance, on calls in a row of different shapes and precisions, the
  largest case first (n = 128, s = 512 fills the static array exactly);
* allocates nothing: the high-water mark of the device's default memory pool
  (the stream-ordered allocator the allocating entry point draws from) does
  not move, while the allocating call, the positive control, raises it;
* rejects sizes beyond its array and a stream of another device.

This file is collected last so a failure here comes after every other test
has run."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2606_18411_gb300 import inputs

pytestmark = pytest.mark.gpu

CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8   # CUmemPool_attribute (cuda.h)
CU_MEMPOOL_ATTR_USED_MEM_CURRENT = 7


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


class DefaultPool:
    """The current device's default memory pool through the driver API."""

    def __init__(self, torch):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)   # resets the high-water mark to the memory in use now
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(z)) == 0


def _noalloc(torch, lib, M, Y, prec):
    s, n = Y.shape
    Rs = M.empty_colmajor(n, n)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.mrcqr_sketch_qr_noalloc(n, s, Y.data_ptr(), M.PREC[prec], Rs.data_ptr(), stream)
    assert rc == 0
    return Rs


# largest first (the whole static array), then smaller shapes and other precisions
CASES = [(128, 512, "fp64", 1), (128, 512, "fp16", 2), (64, 128, "fp64", 3), (100, 200, "fp32", 4),
         (1, 2, "bf16", 5)]


def test_noalloc_matches_allocating_call_and_oracle(env):
    torch, lib, M = env
    for n, s, prec, seed in CASES:
        Yh = inputs.gaussian(s, n, seed=seed) * np.logspace(0, -6, n)[None, :]
        Y = M.to_colmajor(Yh)
        got = _noalloc(torch, lib, M, Y, prec).cpu().numpy()
        ref = M.sketch_qr(Y, prec).cpu().numpy()
        torch.cuda.synchronize()
        # the same kernels on the same input: bit for bit
        np.testing.assert_array_equal(got, ref)
        # and the oracle's Householder QR of Y: column-scaled Gaussian, columnwise ~ u_p
        # (FP16/BF16/FP32 sketches are factored in FP32, the FP64 sketch in FP64)
        tol = 1e-12 if prec == "fp64" else 1e-4
        want = O.householder_qr(Yh)
        colerr = np.linalg.norm(got - want, axis=0) / np.linalg.norm(want, axis=0)
        assert colerr.max() <= tol, (n, s, prec, colerr.max())
        np.testing.assert_array_equal(np.tril(got, -1), 0)
        assert np.all(np.diag(got) > 0)


def test_noalloc_allocates_nothing(env):
    torch, lib, M = env
    pool = DefaultPool(torch)
    Yh = inputs.gaussian(512, 128, seed=9)
    Y = M.to_colmajor(Yh)
    _noalloc(torch, lib, M, Y, "fp64")      # first call in this context done (address looked up)
    torch.cuda.synchronize()
    for prec in ("fp64", "fp32"):
        base = pool.get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)
        pool.reset_high()
        _noalloc(torch, lib, M, Y, prec)
        torch.cuda.synchronize()
        assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) == base, prec
    # positive control: the allocating entry point draws its workspace from this pool
    base = pool.get(CU_MEMPOOL_ATTR_USED_MEM_CURRENT)
    pool.reset_high()
    M.sketch_qr(Y, "fp64")
    torch.cuda.synchronize()
    assert pool.get(CU_MEMPOOL_ATTR_USED_MEM_HIGH) > base


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, lib, M = env
    stream = torch.cuda.current_stream().cuda_stream
    Y = M.empty_colmajor(600, 129)
    Rs = M.empty_colmajor(129, 129)
    assert lib.mrcqr_sketch_qr_noalloc(129, 600, Y.data_ptr(), 3, Rs.data_ptr(), stream) == 1
    Y2 = M.empty_colmajor(513, 64)
    Rs2 = M.empty_colmajor(64, 64)
    assert lib.mrcqr_sketch_qr_noalloc(64, 513, Y2.data_ptr(), 3, Rs2.data_ptr(), stream) == 1
    # still usable after the rejections
    Yh = inputs.gaussian(64, 32, seed=11)
    got = _noalloc(torch, lib, M, M.to_colmajor(Yh), "fp64").cpu().numpy()
    want = O.householder_qr(Yh)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
