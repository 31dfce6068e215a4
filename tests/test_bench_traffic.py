"""bench.py's DRAM-traffic lookup (host logic, no GPU): a figure from a committed ncu capture is
reported only for the workload it was captured on and only while the library sources still hash
to the value recorded beside it."""
import os

import bench


def fake_tree(tmp_path, src="kernel v1"):
    csrc = tmp_path / "paper_1302_4000_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cuh").write_text(src)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_traffic_applies_to_its_workload_and_sources_only(tmp_path, monkeypatch):
    csrc = fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.csrc_hash()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment line\n"
        f"pairs_tc_rot {h} 5000 300 621807104 summary.md\n"
        f"bwd_rot {'0' * 64} 5000 300 123 summary.md\n")
    assert bench.traffic_for("pairs_tc_rot", 5000, 300) == 621807104.0
    assert bench.traffic_for("pairs_tc_rot", 2000, 300) is None  # another N
    assert bench.traffic_for("pairs_tc_rot", 5000, 150) is None  # another L
    assert bench.traffic_for("bwd_rot", 5000, 300) is None  # taken from other sources
    assert bench.traffic_for("cmo_tc", 5000, 300) is None  # never captured
    (csrc / "k.cuh").write_text("kernel v2")  # any source change retires every figure
    assert bench.traffic_for("pairs_tc_rot", 5000, 300) is None


def test_traffic_missing_file_is_none(tmp_path, monkeypatch):
    fake_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert not os.path.exists(tmp_path / "profiles" / "traffic.txt")
    assert bench.traffic_for("pairs_tc_rot", 5000, 300) is None
