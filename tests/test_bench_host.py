"""Host-side arithmetic and bookkeeping of bench.py (CPU only)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_of_the_wide_pair():
    # wide CSC, FP32 values and vectors, int32 indices: Z (4 + 4) + (n + 1) 4 + n 4 + m 4 per product
    m, n, z = 20_000, 5_000_000, 200_286_304
    b_spmv, b_spvtm = bench.pair_bytes(m, n, z)
    assert b_spmv == b_spvtm == 8 * z + 4 * (n + 1) + 4 * n + 4 * m
    assert abs(b_spmv - 1.6423e9) < 1e6  # 1.642 GB per product
    assert bench.pair_bytes(m, n, z, sv=2)[0] == 6 * z + 4 * (n + 1) + 4 * n + 4 * m  # BF16 values


def test_whole_job_value_counts_every_replica():
    assert bench.whole_job_gbs(1e9, 10, 1, 10.0) == 1000.0
    assert bench.whole_job_gbs(1e9, 10, 4, 10.0) == 4000.0


def test_committed_traffic_is_used_only_for_the_kernel_source_workload_and_order_it_was_taken_on(tmp_path,
                                                                                                   monkeypatch):
    entry = {"bytes_per_launch": 123, "source_hash": bench.kernel_source_hash(), "workload": "w",
             "nonzero_order": "bank"}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps({"chunk_scatter": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the source hash is computed from the real kernel sources
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: entry["source_hash"])
    assert bench.ncu_traffic("chunk_scatter", "w", "bank") == 123
    assert bench.ncu_traffic("chunk_scatter", "w", "stored") is None
    assert bench.ncu_traffic("chunk_scatter", "other", "bank") is None
    assert bench.ncu_traffic("chunk_segdot", "w", "bank") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.ncu_traffic("chunk_scatter", "w", "bank") is None


def test_committed_traffic_is_close_to_the_algorithmic_bytes():
    """The DRAM bytes per launch in profiles/dram_traffic.json lie within a few percent of the
    algorithmic bytes (more would mean re-reads).  Skipped once the kernel sources have changed
    since the capture (the bench then reports the traffic as null)."""
    d = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    b_spmv, _ = bench.pair_bytes(20_000, 5_000_000, 200_286_304)
    for name, e in d.items():
        if e["source_hash"] != bench.kernel_source_hash():
            pytest.skip("kernel sources changed since the capture")
        assert e["workload"] == bench.WORKLOAD
        assert 0.95 * b_spmv < e["bytes_per_launch"] < 1.10 * b_spmv, name
