"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; argument checks reject bad calls before anything touches a GPU
(runs without a GPU)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_18411_gb300 import build, _lib
    build.build()
    return _lib.load()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(mrcqr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("mrcqr_factor", "mrcqr_factor_batched", "mrcqr_factor_ex", "mrcqr_get_last_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2606_18411_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.SIGNATURES)


def test_version_and_status_strings(lib):
    assert lib.mrcqr_version() >= 10000
    assert lib.mrcqr_status_string(0) == b"ok"
    assert b"breakdown" in lib.mrcqr_status_string(2).lower()


def test_invalid_arguments_rejected_before_launch(lib):
    P = ctypes.c_void_p
    fake_a, fake_q, fake_r = P(0x10000), P(0x20000000), P(0x40000000)
    # null pointers
    assert lib.mrcqr_factor(100, 4, None, 100, fake_q, 100, fake_r, 3, 0, None) == 1
    # n > m / s > m
    assert lib.mrcqr_factor(6, 4, fake_a, 6, fake_q, 6, fake_r, 3, 0, None) == 1
    # lda < m
    assert lib.mrcqr_factor(100, 4, fake_a, 50, fake_q, 100, fake_r, 3, 0, None) == 1
    # n too large
    assert lib.mrcqr_factor(1 << 20, 1024, fake_a, 1 << 20, fake_q, 1 << 20, fake_r, 3, 0, None) == 1
    # bad precision
    assert lib.mrcqr_factor(100, 4, fake_a, 100, fake_q, 100, fake_r, 9, 0, None) == 1
    # A aliasing Q
    assert lib.mrcqr_factor(100, 4, fake_a, 100, fake_a, 100, fake_r, 3, 0, None) == 1
    assert lib.mrcqr_sample_rows(10, 11, 0, fake_a, None) == 1
    assert lib.mrcqr_signs(0, 0, fake_a, None) == 1


def test_transform_and_estimator_arguments_rejected_before_launch(lib):
    from paper_2606_18411_gb300 import _lib
    P = ctypes.c_void_p
    fake_a, fake_q, fake_r, fake_o = P(0x10000), P(0x20000000), P(0x40000000), P(0x60000000)
    # the real FFT has floor(m/2) + 1 bins: 51 of m = 100 fit, 52 do not; no transform 3
    assert lib.mrcqr_sample_transform_rows(100, 52, 1, 0, fake_o, None) == 1
    assert lib.mrcqr_sample_transform_rows(100, 51, 3, 0, fake_o, None) == 1
    assert lib.mrcqr_sample_transform_rows(100, 101, 0, 0, fake_o, None) == 1
    # Re + Im rows: 2c at most 8192
    assert lib.mrcqr_sketch_transform(1 << 16, 8, fake_a, 1 << 16, 4097, 2, 0, 0, 0, fake_o, None) == 1
    assert lib.mrcqr_sketch_transform(1 << 16, 8, fake_a, 1 << 16, 64, 2, 7, 0, 0, fake_o, None) == 1   # precision
    # factor_ex: s_factor * n bins beyond floor(m/2) + 1 with the real FFT
    o = _lib.Opts(s_factor=3, check=1, escalate=1, sketch_variant=0, ortho_tol=0.0, stats_device=None,
                  fp64_products=0, transform=1)
    assert lib.mrcqr_factor_ex(200, 40, fake_a, 200, fake_q, 200, fake_r, 40, 0, 0, ctypes.byref(o), None) == 1
    o.transform = 5
    assert lib.mrcqr_factor_ex(1 << 12, 8, fake_a, 1 << 12, fake_q, 1 << 12, fake_r, 8, 0, 0, ctypes.byref(o), None) == 1
    # regime estimates: method, m < n, lda < m, null output
    assert lib.mrcqr_regime_estimate(64, 8, fake_a, 64, 2, 0, fake_o, None) == 1
    assert lib.mrcqr_regime_estimate(4, 8, fake_a, 64, 0, 0, fake_o, None) == 1
    assert lib.mrcqr_regime_estimate(64, 8, fake_a, 63, 1, 0, fake_o, None) == 1
    assert lib.mrcqr_regime_estimate(64, 8, fake_a, 64, 1, 0, None, None) == 1
    # bounded-wait hook: polls out of range
    assert lib.mrcqr_debug_wait_timeout(0, fake_o, None) == 1
    assert lib.mrcqr_debug_wait_timeout((1 << 20) + 1, fake_o, None) == 1
