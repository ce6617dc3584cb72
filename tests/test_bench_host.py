"""Host logic of bench.py that needs no GPU: the comparison of two partitions
(used against the stored oracle digest of the 8192^2 map) and the choice of
the committed DRAM-traffic capture that a bench line's roofline uses."""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_partition_mismatch_equal_partitions_up_to_relabelling():
    a = np.array([0, 0, 1, 2, 2, 2])
    b = np.array([5, 5, 3, 9, 9, 9])
    assert bench.partition_mismatch(a, b) == (0, 0, 0)


def test_partition_mismatch_one_split_group():
    # seeding components 3..5 form one group in a and two groups in b
    a = np.array([0, 0, 1, 2, 2, 2])
    b = np.array([0, 0, 1, 2, 2, 7])
    nc, ga, gb = bench.partition_mismatch(a, b)
    assert (nc, ga, gb) == (3, 1, 2)
    # symmetric in the roles of the two partitions
    assert bench.partition_mismatch(b, a) == (3, 2, 1)


def test_partition_mismatch_crossing_groups():
    # {0,1},{2,3} against {0},{1,2},{3}: every component is in a group that
    # is not a group of the other partition
    a = np.array([0, 0, 1, 1])
    b = np.array([0, 1, 1, 2])
    assert bench.partition_mismatch(a, b) == (4, 2, 3)


def _fake_root(tmp_path, src_text, captures, sha=None):
    csrc = tmp_path / "paper_2510_11508_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = sha or hashlib.sha256(src_text.encode()).hexdigest()
    caps = {c["workload"]: c for c in captures}
    (prof / "k_x_traffic.json").write_text(json.dumps({"source_sha256": h, "captures": caps}))


def test_traffic_capture_of_largest_map_not_larger(tmp_path, monkeypatch):
    caps = [{"workload": "small", "grid_px": 100, "dram_bytes_per_px_iter": 60.0},
            {"workload": "big", "grid_px": 1000, "dram_bytes_per_px_iter": 110.0}]
    _fake_root(tmp_path, "kernel source", caps)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_px_iter("k_x", "k.cu", 5000) == (110.0, "big")
    assert bench.traffic_per_px_iter("k_x", "k.cu", 1000) == (110.0, "big")
    assert bench.traffic_per_px_iter("k_x", "k.cu", 999) == (60.0, "small")
    assert bench.traffic_per_px_iter("k_x", "k.cu", 10) == (60.0, "small")


def test_traffic_is_none_once_the_kernel_changed(tmp_path, monkeypatch):
    caps = [{"workload": "small", "grid_px": 100, "dram_bytes_per_px_iter": 60.0}]
    _fake_root(tmp_path, "kernel source", caps, sha="0" * 64)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_px_iter("k_x", "k.cu", 5000) == (None, None)
    assert bench.traffic_per_px_iter("k_missing", "k.cu", 5000) == (None, None)


def test_committed_traffic_record_matches_the_fill_kernel():
    """The committed captures were taken on the fill kernel as it is now, and
    the 8192^2 line takes the 4096^2 capture."""
    tpi, cap = bench.traffic_per_px_iter("k_pcg_mg", "ni_mg.cu", 8192 * 8192)
    assert cap == "c4_4096_persp" and 90.0 < tpi < 130.0
    tpi, cap = bench.traffic_per_px_iter("k_pcg_mg", "ni_mg.cu", 2048 * 2048)
    assert cap == "c3_2048_persp" and 50.0 < tpi < 90.0
