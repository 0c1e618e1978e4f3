"""Host-side arithmetic of bench.py's roofline objects: the achieved rate and
fraction from algorithmic bytes and a time, the DRAM fields from captured
traffic, and captured traffic that is dropped once its kernel's source no
longer matches the capture."""
import hashlib

import bench


def test_roofline_fractions():
    r = bench.roofline("hbm", 6.0e9, 2.0e-3, 6000.0, "GB/s", "k", traffic=9.0e9)
    assert r["achieved"] == 3000.0 and r["frac"] == 0.5
    assert r["dram_gbs"] == 4500.0 and r["dram_frac"] == 0.75
    assert r["traffic"] == 9.0e9 and r["algorithmic"] == 6.0e9 and r["seconds"] == 2.0e-3
    t = bench.roofline("tensor", 3.0e12, 1.0e-2, 1500.0, "TFLOP/s", "k")
    assert t["achieved"] == 300.0 and t["frac"] == 0.2
    assert t["traffic"] is None and "dram_gbs" not in t


def test_measured_traffic_follows_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    sha = hashlib.sha1(src.read_bytes()).hexdigest()[:12]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC", {"k": {"src": "kernel.cu", "sha1": sha, "bytes_per_unit": 2.5}})
    assert bench.measured_traffic("k", 4e6) == 1e7  # scaled by the units of the launch
    assert bench.measured_traffic("other", 4e6) is None
    src.write_bytes(b"__global__ void k() { /* changed */ }\n")
    assert bench.measured_traffic("k", 4e6) is None  # the counters no longer describe the kernel


def test_every_traffic_entry_names_a_kernel_source():
    for name, t in bench.TRAFFIC.items():
        assert t["src"].startswith("paper_2211_02753_b300/csrc/") and t["src"].endswith(".cu"), name
        assert len(t["sha1"]) == 12 and t["bytes_per_unit"] > 0, name
