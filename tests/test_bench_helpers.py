"""Host logic of bench.py's roofline entry (no GPU): matching a committed ncu summary to
the kernel's current device code, and the DRAM-traffic model of the average launch."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import pytest  # noqa: E402


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


class _FakeSolver:
    """Stands in for paper_2510_12731_gb300.Solver: fixed statistics, every column
    converged, no device."""

    def __init__(self, **opts):
        self.opts = opts
        self.natoms = 0
        self.model = 0

    def set_structure(self, model, xyz, type_idx, types):
        self.natoms = len(xyz)

    def solve_device(self, omega_ev, pol_dirs, alpha_ib=None, e0=1.0, d_alpha=None, d_q=None,
                     d_mu=None, d_relres=None, stream=None):
        if d_relres is not None:
            d_relres.zero_()
        return True

    def alloc_outputs(self, F, P, want_q=True, want_mu=True, empty=None):
        import numpy as np
        return {"alpha": np.zeros((F, 3, P), complex), "rel_residual": np.zeros((F, P)),
                "status": np.zeros((F, P), np.int32)}

    def solve(self, omega_ev, pol_dirs, alpha_ib=None, out=None):
        return out

    def stats(self):
        return {"kernel_launches": 100, "setup_launches": 10, "matvec_ms": 5.0,
                "matvec_launches": 10, "matvec_flops": 4.0 * 7119 ** 2 * 300 * 10,
                "total_iters": 10, "graph_launches": 0}

    def close(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def test_gpu_arm_emits_the_contract_line(monkeypatch, capsys):
    """run_ours end to end on the CPU: torch's CUDA calls and the solver replaced by
    stand-ins; the JSON line carries every key of the bench contract."""
    import json
    import torch
    import paper_2510_12731_gb300 as pkg

    class _Ev:
        t = 0.0

        def __init__(self, enable_timing=True):
            self.at = None

        def record(self):
            _Ev.t += 1.0
            self.at = _Ev.t

        def elapsed_time(self, other):
            return 1000.0 * (other.at - self.at)

    real_empty = torch.empty
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Event", _Ev)
    monkeypatch.setattr(torch, "device", lambda *a: "cpu")
    monkeypatch.setattr(torch, "empty",
                        lambda *a, **k: real_empty(*a, **{x: y for x, y in k.items()
                                                          if x not in ("pin_memory",)}))
    monkeypatch.setattr(pkg, "Solver", _FakeSolver)
    monkeypatch.setattr(bench.ClockSampler, "start", lambda self: None)
    args = bench.argparse.Namespace(
        gpus=1, steps=2, warmup=1, impl="ours", workload="na_sphere40", precision="fp32",
        mode=None, restart_m=0, gs_passes=1, basis="auto", graphs=False, inner_tol=None,
        e2e_steps=1, cpu_freqs=1, no_cpu_baseline=True, p0_cols=0, serve_requests=2,
        serve_nmax=600, serve_slots=1)
    assert bench.run_ours(args, 0, 1, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "clocks", "e2e", "gpu_launches", "roofline", "cpu_baseline"):
        assert k in line, k
    assert line["points_per_step"] == 300          # 100 w x 3 pols, all converged
    assert line["gpu_launches"] == 2 * 110
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    assert set(line["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert line["config"]["workload"] == "na_sphere_r40A_wfq"
    assert line["dtype"] == bench.DTYPES["fp32"]


def test_reference_arm_line(capsys):
    """The reference arm (the CPU oracle) on the 791-atom workload: one JSON line with
    impl, cpu_baseline and an e2e entry whose value is the line's own."""
    import json
    args = bench.argparse.Namespace(gpus=1, steps=1, warmup=1, workload="ag_sphere",
                                    cpu_freqs=1, ref_budget_s=240.0)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["steps"] == 1
    assert line["e2e"]["value"] == line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert bench.run_reference(args, 1, 2) == 0          # other ranks exit without work


def test_reference_arm_stops_at_its_budget(capsys, monkeypatch):
    """With samples slower than the budget allows, the arm times one step (never zero)
    and reports how many it timed out of those requested."""
    import json
    calls = []

    def fake_sample(wl, n_freq=1):
        calls.append(wl.name)
        return 50.0, 3

    monkeypatch.setattr(bench, "_oracle_sample", fake_sample)
    args = bench.argparse.Namespace(gpus=1, steps=20, warmup=5, workload="ag_sphere",
                                    cpu_freqs=1, ref_budget_s=60.0)
    assert bench.run_reference(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["steps"] == 1 and line["steps_requested"] == 20
    assert line["value"] == pytest.approx(3 / 50.0)
    assert len(calls) == 5 + 1                     # warm-up samples, then one timed step
