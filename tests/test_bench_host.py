"""Host logic of bench.py that needs no GPU: workload selection, the traffic
records and their invalidation, and the oracle's bounded sample."""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import gen  # noqa: E402


def test_rmat_scale_override():
    w = bench.select_workload("rmat26", 16)
    assert (w["scale"], w["n"], w["workload"]) == (16, 1 << 16, "rmat_s16_ef16")
    assert w["oracle_draws"] == 16 << 16  # capped by the number of draws
    assert bench.WORKLOADS["rmat26"]["scale"] == 26  # the table itself is unchanged
    assert bench.select_workload("chung_lu", 16) == bench.WORKLOADS["chung_lu"]  # ignored elsewhere


def _records(tmp_path, text):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "a.cu").write_text(text)
    sha = hashlib.sha1(b"kernel source").hexdigest()[:12]
    rec = {"records": [{"kernel": "k_x", "workload": "w1", "sources": ["a.cu"], "sources_sha1_12": sha,
                        "dram_bytes": 123}]}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))


def test_traffic_record_matches_workload_kernel_and_source(tmp_path, monkeypatch):
    _records(tmp_path, "kernel source")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("w1", "k_x") == 123.0
    assert bench.recorded_traffic("w2", "k_x") is None
    assert bench.recorded_traffic("w1", "k_y") is None


def test_traffic_record_dropped_when_the_source_changed(tmp_path, monkeypatch):
    _records(tmp_path, "kernel source, edited")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("w1", "k_x") is None


def test_rmat_oracle_sample_is_the_canonical_prefix(monkeypatch):
    w = bench.select_workload("rmat26", 12)
    monkeypatch.setattr(bench, "WORKLOAD", dict(w, oracle_draws=1 << 14))
    draws = gen.rmat_draws(12, 16, seed=1)
    canon, p, what = bench.oracle_sample(draws, w["n"])
    assert p == min(w["p_sweep"]) and "first 16384" in what
    u = np.minimum(draws[:1 << 14, 0], draws[:1 << 14, 1]).astype(np.uint64)
    v = np.maximum(draws[:1 << 14, 0], draws[:1 << 14, 1]).astype(np.uint64)
    keys = np.unique((u << np.uint64(32) | v)[u != v])
    assert np.array_equal(canon[:, 0].astype(np.uint64) << np.uint64(32) | canon[:, 1], keys)


def test_default_workload_is_the_largest_graph():
    """The default run (what the driver times) is R-MAT scale 26 with the
    batched and served comparisons as extra keys."""
    assert bench.DEFAULT_WORKLOAD == "rmat26"
    old = sys.argv
    try:
        sys.argv = ["bench.py"]
        args = bench.parse_args()
    finally:
        sys.argv = old
    assert args.workload == "rmat26" and args.gpus == 1 and not args.no_extras
    w = bench.WORKLOADS["rmat26"]
    assert (w["scale"], w["edge_factor"], w["p_sweep"]) == (26, 16, [1.0, 0.05])


def test_traffic_record_scaled_from_a_smaller_case(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "a.cu").write_text("kernel source")
    sha = hashlib.sha1(b"kernel source").hexdigest()[:12]
    rec = {"records": [{"kernel": "k_x", "workload": "big", "sources": ["a.cu"], "sources_sha1_12": sha,
                        "dram_bytes": 80, "algorithmic_bytes": 100, "scale_by_algorithmic_bytes": True}]}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("big", "k_x", 1000.0) == 800.0
    assert bench.recorded_traffic("big", "k_x") is None
