"""The bench's roofline traffic (bench.ncu_traffic): the per-particle DRAM
bytes of a capture scaled to the launch by its particle count, looked up by
kernel / workload / precision / cell order, and null once the kernel's
sources differ from the captured build."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write(tmp_path, h):
    (tmp_path / "profiles").mkdir()
    d = {"kernel_hash": h, "kernels": {
        "k_cellpass/batch256/mixed": {"bytes_per_particle": 66.0},
        "k_cellpass/batch256/mixed/hilbert": {"bytes_per_particle": 67.0},
        "k_cellpass/dimer32/mixed": {"bytes_per_launch": 12345}}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps(d))


def test_traffic_scaled_by_particles_and_keyed_by_order(tmp_path, monkeypatch):
    _write(tmp_path, "h1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda kernel="k_cellpass": "h1")
    assert bench.ncu_traffic("k_cellpass", "batch256", "mixed", 1000) == 66000
    assert bench.ncu_traffic("k_cellpass", "batch256", "mixed", 1000, "hilbert") == 67000
    assert bench.ncu_traffic("k_cellpass", "dimer32", "mixed", 1000) == 12345
    assert bench.ncu_traffic("k_cellpass", "batch256", "fp64", 1000) is None
    assert bench.ncu_traffic("k_cellpass", "poiseuille128", "mixed", 1000) is None


def test_traffic_null_for_another_build(tmp_path, monkeypatch):
    _write(tmp_path, "h1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda kernel="k_cellpass": "h2")
    assert bench.ncu_traffic("k_cellpass", "batch256", "mixed", 1000) is None


def test_committed_capture_names_a_hash_of_the_kernel_sources():
    d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    assert len(d["kernel_hash"]) == 16 and set(d["kernel_hash"]) <= set("0123456789abcdef")
    for key, e in d["kernels"].items():
        assert key.startswith("k_cellpass/")
        # at least the algorithmic 64 bytes of a mixed record read and written
        assert 64.0 <= e["bytes_per_particle"] < 2 * 64.0
