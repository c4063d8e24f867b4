"""Host-side pieces of bench.py's JSON line, checked without a GPU.

The roofline's `traffic` comes from committed ncu counters and must turn null
as soon as the kernel source differs from the one the counters were taken on;
the algorithmic bytes per cell-direction follow from the path's minimum
traffic (N_H store per cell-direction; density read, screening store and the
coarse levels per leaf).
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_per_cell_direction():
    # 4 B of N_H per cell-direction; 4 B density + 4 B screening factor + 4/7 B of
    # coarse levels (levels 0..L-1 hold 1/7 of the leaves) per leaf
    assert bench.algo_bytes_per_cell_dir(48) == pytest.approx(4.0 + (8.0 + 4.0 / 7.0) / 48, rel=1e-15)
    assert bench.algo_bytes_per_cell_dir(12) == pytest.approx(4.0 + (8.0 + 4.0 / 7.0) / 12, rel=1e-15)
    # 256^3 x 48: 805.3 M cell-directions, 3.365 GB
    assert bench.algo_bytes_per_cell_dir(48) * (256 ** 3) * 48 == pytest.approx(3.365e9, rel=1e-3)


def test_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = tmp_path / "paper_1410_0624_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "leaf_tc.cu").write_text("kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench._source_hash("leaf_tc.cu")
    entry = {"dram_bytes_per_launch": 1234, "source_sha256_16": h}
    (prof / "traffic.json").write_text(json.dumps({"leaf_tc/L8/nd48": entry}))
    # the BF16 leaf kind maps to the tensor-core leaf kernel's entry
    assert bench.measured_traffic("leaf", 8, 48, "bf16") == 1234
    assert bench.measured_traffic("leaf", 7, 48, "bf16") is None        # no entry for that size
    # a per-step figure (several launches a step) takes precedence
    entry["dram_bytes_per_step"] = 5678
    (prof / "traffic.json").write_text(json.dumps({"leaf_tc/L8/nd48": entry}))
    assert bench.measured_traffic("leaf", 8, 48, "bf16") == 5678
    # the kernel changed since the counters were taken: no traffic figure
    (src / "leaf_tc.cu").write_text("kernel v2\n")
    assert bench.measured_traffic("leaf", 8, 48, "bf16") is None


def test_committed_traffic_entries_name_their_kernels():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        tr = json.load(f)
    for key, e in tr.items():
        kind = key.split("/")[0]
        assert kind in bench.KERNEL_SOURCES, key
        assert e["dram_read"] + e["dram_write"] == pytest.approx(e["dram_bytes_per_launch"], abs=2)
        assert len(e["source_sha256_16"]) == 16
