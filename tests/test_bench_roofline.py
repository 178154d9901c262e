"""Host logic of the bench's roofline: the algorithmic work per stage and the
committed DRAM traffic, which is used only while the kernel's source matches
the capture it came from."""
from __future__ import annotations

import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_stage_work_is_the_algorithmic_count():
    m, n = 1 << 20, 512
    b, f64, tf = bench.stage_work("trsm", m, n)
    assert b == 16.0 * m * n                      # A read once, W written once
    assert f64 == 1.0 * m * n * n                 # one triangular solve
    assert tf == 36.0 * m * n * (n - 16)          # 36 digit-pair products per multiply-add of the updates
    assert bench.stage_work("syrk", m, n)[0] == 8.0 * m * n
    assert bench.stage_work("finalize", m, n)[0] == 16.0 * m * n
    assert bench.stage_work("sketch", m, n)[0] == 8.0 * m * n
    assert bench.stage_work("chol", m, n) is None


def test_committed_traffic_is_read_while_the_source_matches(tmp_path, monkeypatch):
    d = json.load(open(bench.PROFILE_TRAFFIC))
    src = os.path.join(ROOT, "paper_2606_18411_gb300", "csrc", d["trsm"]["source"])
    d["trsm"]["source_sha256"] = hashlib.sha256(open(src, "rb").read()).hexdigest()
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(d))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(p))
    ent = bench.load_traffic("trsm")
    assert ent is not None and ent["bytes_per_row"] == d["trsm"]["bytes_per_row"]


def test_traffic_is_dropped_when_the_source_changes(tmp_path, monkeypatch):
    d = json.load(open(bench.PROFILE_TRAFFIC))
    d["trsm"]["source_sha256"] = hashlib.sha256(b"another kernel").hexdigest()
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(d))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(p))
    assert bench.load_traffic("trsm") is None
    assert bench.load_traffic("no_such_kernel") is None
