"""Host logic of bench.py's roofline entry (no GPU): matching a committed ncu summary to
the kernel's current device code, and the DRAM-traffic model of the average launch."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_tc_profile_matches_current_device_code():
    """The committed tensor-core summary was captured on the current device code, so its
    DRAM / algorithmic ratio is used; the host launcher below the device part does not
    enter the hash."""
    text = open(os.path.join(ROOT, "profiles", "k_tc_gemm_fp16split.md")).read()
    assert bench.kernel_source_sha("k_gemm_tc.cu") in text
    ratio = bench._profile_ratio("k_gemm_tc.cu", "k_tc_gemm_fp16split.md")
    assert ratio is not None and 1.0 <= ratio < 1.5


def test_device_part_hash_ignores_host_code(tmp_path, monkeypatch):
    src = open(os.path.join(ROOT, "paper_2510_12731_gb300", "csrc", "k_gemm_tc.cu"), "rb").read()
    marker = bench.DEVICE_PART_END["k_gemm_tc.cu"]
    head, tail = src.split(marker, 1)
    d = tmp_path / "paper_2510_12731_gb300" / "csrc"
    d.mkdir(parents=True)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (d / "k_gemm_tc.cu").write_bytes(head + marker + tail + b"\n// host-side change\n")
    h_host = bench.kernel_source_sha("k_gemm_tc.cu")
    (d / "k_gemm_tc.cu").write_bytes(head + b"// device-side change\n" + marker + tail)
    h_dev = bench.kernel_source_sha("k_gemm_tc.cu")
    monkeypatch.setattr(bench, "ROOT", ROOT)
    assert h_host == bench.kernel_source_sha("k_gemm_tc.cu")
    assert h_dev != h_host


def test_tensor_roofline_traffic_model():
    """traffic = ratio x (4 np^2 + 16 np B) for the average launch; achieved / peak."""
    n_u = 19931
    b = 600
    flops = 4.0 * n_u * n_u * b
    r = bench._roofline("fp16split", "materialised", flops, 1e-3, 10, n_u=n_u)
    np_ = 19968
    ratio = bench._profile_ratio("k_gemm_tc.cu", "k_tc_gemm_fp16split.md")
    assert abs(r["traffic"] - ratio * (4.0 * np_ * np_ + 16.0 * np_ * b)) < 1.0
    assert abs(r["achieved"] - flops / 1e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["bound"] == "tensor"


def test_fp64_and_fp32_rooflines_use_alu_peaks():
    r64 = bench._roofline("fp64", "materialised", 1e12, 1.0, 1)
    assert r64["bound"] == "alu" and r64["peak"] == bench.FP64_PEAK_TFLOPS
    r32 = bench._roofline("fp32", "materialised", 1e12, 1.0, 1)
    assert r32["bound"] == "alu" and abs(r32["peak"] - 152 * 128 * 2 * 2.070e9 / 1e12) < 1e-9


def test_fp32_gemm_profile_matches_and_models_traffic():
    """The FP32 GEMM summary matches the current code of that kernel (the FP64 kernels
    sharing its file are outside the hashed span); traffic = ratio x algorithmic bytes."""
    ratio = bench._profile_ratio("k_gemm_simt.cu", "k_sgemm_fp32.md")
    assert ratio is not None and 0.9 < ratio < 1.2
    n_u, b = 22052, 450
    r = bench._roofline("fp32", "materialised", 4.0 * n_u * n_u * b, 1e-2, 5, n_u=n_u)
    np_ = 22144
    assert abs(r["traffic"] - ratio * (4.0 * np_ * np_ + 16.0 * np_ * b)) < 1.0
