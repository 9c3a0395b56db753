"""Host logic of bench.py (CPU): the roofline arithmetic of each form and the
DRAM-traffic record, which counts only while the kernel source is unchanged."""
import hashlib
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 8000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1600.0,
         "source": "test", "sm_max_mhz": 2000.0}


def test_roofline_gemm_counts_four_k_flops_per_evaluation():
    # 1e12 evaluations with K = 10 in 25 ms: 4 * 10 * 1e12 / 0.025 s = 1.6e15 flop/s
    r = bench.roofline("gemm", 10, 1e12, 25.0, PEAKS, None)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(1600.0)
    assert r["frac"] == pytest.approx(1.0)


def test_roofline_permblock_counts_two_lane_ops_per_evaluation():
    # peak: 152 SMs x 128 lanes x 2,000 MHz = 38.912 T lane-op/s
    r = bench.roofline("permblock", 4, 1e12, 100.0, PEAKS, None)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert r["achieved"] == pytest.approx(2e12 / 0.1 / 1e12)


def test_roofline_brute_counts_four_bytes_per_evaluation():
    r = bench.roofline("brute", 4, 1e12, 500.0, PEAKS, 1.5e12)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(4e12 / 0.5 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 8000.0)
    assert r["traffic"] == 1.5e12


def _tree(tmp_path, src_text, record):
    csrc = tmp_path / "paper_2505_04556_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_gemm.cu").write_text(src_text)
    (tmp_path / "profiles").mkdir()
    if record is not None:
        (tmp_path / "profiles" / "traffic.txt").write_text(record)
    return hashlib.sha1(src_text.encode()).hexdigest()[:12]


def test_traffic_record_applies_only_to_the_measured_source(tmp_path, monkeypatch):
    sha = _tree(tmp_path, "// kernel v1\n", None)
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f'form=gemm src_sha={sha} bytes_per_eval=2.0e-02 capture="ncu --metrics x" read_GB=1\n')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch("gemm", 1e12) == pytest.approx(2.0e10)
    # the source changes: the record no longer describes it
    (tmp_path / "paper_2505_04556_gb300" / "csrc" / "k_gemm.cu").write_text("// kernel v2\n")
    assert bench.traffic_per_launch("gemm", 1e12) is None


def test_traffic_record_missing(tmp_path, monkeypatch):
    _tree(tmp_path, "// kernel\n", None)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch("gemm", 1e12) is None



def test_traffic_record_applies_only_to_its_workload(tmp_path, monkeypatch):
    sha = _tree(tmp_path, "// kernel\n", None)
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"form=gemm src_sha={sha} bytes_per_eval=1.0e-02 workload=euclid-100k read_GB=1\n"
        f"form=gemm src_sha={sha} bytes_per_eval=3.0e-03 workload=euclid-20k read_GB=1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_launch("gemm", 1e12, "euclid-100k") == pytest.approx(1.0e10)
    assert bench.traffic_per_launch("gemm", 1e12, "euclid-20k") == pytest.approx(3.0e9)
    assert bench.traffic_per_launch("gemm", 1e12, "jaccard-25k") is None
