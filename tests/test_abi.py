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
