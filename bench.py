"""Benchmark: wFQ spectrum points/s on one GB300 (replicas across GPUs under torchrun).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

One step is the whole hot path on one synthetic structure: staging, neighbour
list / CSR of K, T build, the batched Krylov solve of every (frequency,
polarisation) column with FP64 refinement, and the observables.  A spectrum
point is one column that met the FP64 relative-residual tolerance.

Rank 0 prints ONE JSON line.  ``value`` is timed with CUDA events with the
structure's inputs created on the host and all results left in device memory;
``e2e`` is the same step through the host-buffer call (px_solve), inputs from
pinned host memory and every result copied back, inside the timed region.
``--impl reference`` times the FP64 CPU checker (dense LU) on a bounded sample of
the same workload on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ωFQ spectrum points/s at |Δα|/|α|≤1e-5 vs plain FP64 GPU solve; p50/p99 latency"
UNIT = "points/s"

# FP32 CUDA-core peak of the GB300: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (max SM clock)
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f), "of measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def _roofline(prec, flops_per_launch, avg_launch_s, launches):
    """Roofline entry of the block matvec (the dominant kernel) for the precision used."""
    achieved = flops_per_launch / avg_launch_s / 1e12
    if prec in ("bf16split", "fp16split"):
        peaks, src = _measured_peaks()
        peak = float(peaks["bf16_tflops_sustained"])
        traffic, _ = _profile_traffic("k_gemm_tc.cu", "k_tc_gemm_bf16.md")
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": f"k_tc_gemm (tcgen05 {prec} block matvec, 3 MMAs per product)",
                "peak_source": f"bf16 dense sustained ({src}); algorithmic flops 4 n_u^2 B, "
                               "executed tensor flops are 3x",
                "avg_launch_ms": avg_launch_s * 1e3, "launches": launches}
    traffic, _ = _profile_traffic("k_gemm_simt.cu", "k_sgemm_fp32.md")
    return {"bound": "alu", "achieved": achieved, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_ALU_PEAK_TFLOPS, "traffic": traffic,
            "kernel": "k_sgemm (FP32 CUDA-core block matvec on the materialised T)",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
            "avg_launch_ms": avg_launch_s * 1e3, "launches": launches}


def _workload(name):
    from paper_2510_12731_gb300 import structures as S
    table = {
        "na_ico": S.na_icosahedron_19931,
        "ag_sphere": S.ag_sphere_791,
        "graphene_disk": S.graphene_disk_20nm,
        "ag_rod": S.ag_rod_3x3x10,
        "na_sphere40": S.na_sphere_r40,
    }
    return table[name]()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline traffic
def _profile_traffic(kernel_file, profile_file):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current source of the kernel (the summary records the source's sha256)."""
    path = os.path.join(ROOT, "profiles", profile_file)
    src = os.path.join(ROOT, "paper_2510_12731_gb300", "csrc", kernel_file)
    if not (os.path.exists(path) and os.path.exists(src)):
        return None, None
    text = open(path).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_tr = re.search(r"traffic_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    if not (m_sha and m_tr) or m_sha.group(1) != sha:
        return None, sha
    return float(m_tr.group(1)), sha


# ---------------------------------------------------------------- reference arm
def _oracle_sample(wl, n_freq=1):
    """Time the FP64 CPU checker (dense LU, Eq. 1) on the first n_freq frequencies of
    the workload with every polarisation; returns (seconds, points)."""
    from oracle import model as M
    st = M.structure_from_types(wl.xyz_ang, wl.type_idx, wl.types)
    idx = np.linspace(0, wl.omega_ev.size - 1, n_freq).round().astype(int)
    t0 = time.perf_counter()
    M.solve(st, wl.model, wl.omega_ev[idx], wl.pol_dirs,
            alpha_ib=None if wl.alpha_ib is None else wl.alpha_ib[:, idx])
    dt = time.perf_counter() - t0
    return dt, n_freq * wl.pol_dirs.shape[0]


def _cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    wl = _workload(args.workload)
    for _ in range(args.warmup):
        _oracle_sample(wl, args.cpu_freqs)
    times = []
    pts = 0
    for _ in range(args.steps):
        dt, p = _oracle_sample(wl, args.cpu_freqs)
        times.append(dt)
        pts = p
    per = sum(times) / len(times)
    value = pts / per
    sample = (f"dense LU (numpy/LAPACK) of the full N={wl.natoms} system for {args.cpu_freqs} "
              f"frequency x {wl.pol_dirs.shape[0]} polarisations per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "natoms": wl.natoms, "columns": wl.ncols},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2510_12731_gb300 import Solver

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = _workload(args.workload)
    F, P, N = wl.omega_ev.size, wl.pol_dirs.shape[0], wl.natoms
    opts = dict(precision=args.precision or wl.precision, tol_rel=wl.tol, profile=1,
                restart_m=args.restart_m, gs_passes=args.gs_passes)
    if args.inner_tol:
        opts["inner_tol"] = args.inner_tol
    if args.mode:
        opts["mode"] = args.mode
    solver = Solver(**opts)
    dev = torch.device("cuda", local_rank)
    d_alpha = torch.empty((F, 3, P), dtype=torch.complex128, device=dev)
    d_q = torch.empty((F, P, N), dtype=torch.complex128, device=dev)
    d_rr = torch.empty((F, P), dtype=torch.float64, device=dev)

    def step_device():
        solver.set_structure(wl.model, wl.xyz_ang, wl.type_idx, wl.types)
        ok = solver.solve_device(wl.omega_ev, wl.pol_dirs, wl.alpha_ib, d_alpha=d_alpha, d_q=d_q,
                                 d_relres=d_rr)
        return ok

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step_device()
    barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    mv_ms = 0.0
    mv_n = 0
    mv_flops = 0.0
    converged = 0
    iters = 0
    t_wall0 = time.perf_counter()
    ev0.record()
    for _ in range(args.steps):
        step_device()
        st = solver.stats()
        launches += st["kernel_launches"] + st["setup_launches"]
        mv_ms += st["matvec_ms"]
        mv_n += st["matvec_launches"]
        mv_flops += st["matvec_flops"]
        iters += st["total_iters"]
        converged += int((d_rr <= wl.tol).sum().item())
    ev1.record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    barrier()
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    points_per_step = converged / args.steps
    value = world * points_per_step / (ms / args.steps / 1e3)

    # ---- end to end through the host-buffer call, pinned host memory
    def pinned(shape, dtype):
        t = torch.empty(shape, dtype={np.complex128: torch.complex128, np.float64: torch.float64,
                                      np.int32: torch.int32}[np.dtype(dtype).type], pin_memory=True)
        return t.numpy()

    xyz_p = pinned(wl.xyz_ang.shape, np.float64)
    xyz_p[...] = wl.xyz_ang
    tid_p = pinned(wl.type_idx.shape, np.int32)
    tid_p[...] = wl.type_idx
    out = solver.alloc_outputs(F, P, want_q=True, want_mu=True, empty=lambda s, dtype: pinned(s, dtype))

    def step_e2e():
        solver.set_structure(wl.model, xyz_p, tid_p, wl.types)
        return solver.solve(wl.omega_ev, wl.pol_dirs, wl.alpha_ib, out=out)

    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    step_e2e()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    e2e_pts = 0
    for _ in range(e2e_steps):
        r = step_e2e()
        e2e_pts += int((r["status"] == 0).sum())
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = world * (e2e_pts / e2e_steps) / (e2e_ms / e2e_steps / 1e3)
    h2d = wl.xyz_ang.nbytes + wl.type_idx.nbytes + wl.omega_ev.nbytes + wl.pol_dirs.nbytes + \
        64 * len(wl.types) + (0 if wl.alpha_ib is None else wl.alpha_ib.nbytes)
    d2h = sum(v.nbytes for k, v in out.items() if isinstance(v, np.ndarray)
              and not (k == "sigma_abs" and P != 3))

    # ---- roofline of the dominant kernel (the block matvec)
    prec = opts["precision"]
    avg_launch_s = (mv_ms / mv_n) / 1e3 if mv_n else float("nan")
    flops_per_launch = mv_flops / mv_n if mv_n else float("nan")
    roofline = _roofline(prec, flops_per_launch, avg_launch_s, mv_n)

    # ---- plain FP64 GPU solve (P0): one (frequency, polarisation) column at a time, FP64
    # matvec (GEMV on the FP64 T) and FP64 GMRES, same tolerance; timed on a sample of
    # columns spread over the sweep (lowest frequency included), set-up excluded.
    p0 = None
    if args.p0_cols > 0:
        p0s = Solver(precision="fp64", tol_rel=wl.tol, restart_m=args.restart_m)
        p0s.set_structure(wl.model, wl.xyz_ang, wl.type_idx, wl.types)
        fidx = np.unique(np.linspace(0, F - 1, args.p0_cols).round().astype(int))
        t_tot, n_ok, its = 0.0, 0, 0
        d1 = torch.empty((1, 1), dtype=torch.float64, device=dev)
        for fi in fidx:
            aib = None if wl.alpha_ib is None else wl.alpha_ib[:, fi:fi + 1]
            torch.cuda.synchronize()
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record()
            ok = p0s.solve_device(wl.omega_ev[fi:fi + 1], wl.pol_dirs[:1], aib, d_relres=d1)
            q1.record()
            torch.cuda.synchronize()
            t_tot += q0.elapsed_time(q1) / 1e3
            n_ok += int(ok)
            its += p0s.stats()["total_iters"]
        p0s.close()
        p0 = {"value": n_ok / t_tot, "unit": UNIT, "columns_timed": int(len(fidx)),
              "converged": n_ok, "iters_per_column": its / len(fidx),
              "sample": f"{len(fidx)} columns (w index {fidx.tolist()}, first polarisation), "
                        "each solved alone with FP64 matvec and FP64 GMRES; set-up excluded"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, pts = _oracle_sample(wl, args.cpu_freqs)
        cpu = {"value": pts / dt, "unit": UNIT, "cores": _cores(), "kind": "oracle",
               "sample": f"dense LU of the full N={N} system, {args.cpu_freqs} frequency x {P} "
                         f"polarisations ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": wl.name, "natoms": N, "n_unknowns": N if wl.model == "wfq" else 4 * N,
                       "n_freq": F, "n_pol": P, "columns": F * P, "tol_rel": wl.tol,
                       "precision": prec, "restart_m": args.restart_m, "gs_passes": args.gs_passes,
                       "l2": "no flush: the per-step working set (T, Krylov basis) is far larger than L2",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk, "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                                   "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "p0_fp64_gpu": p0, "vs_p0": (value / world / p0["value"]) if p0 else None,
            "points_per_step": points_per_step, "iters_per_step": iters / args.steps,
            "wall_s": wall,
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="na_ico")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--mode", default=None)
    ap.add_argument("--restart-m", dest="restart_m", type=int, default=100)
    ap.add_argument("--gs-passes", dest="gs_passes", type=int, default=1)
    ap.add_argument("--inner-tol", dest="inner_tol", type=float, default=None)
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=2)
    ap.add_argument("--cpu-freqs", dest="cpu_freqs", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--p0-cols", dest="p0_cols", type=int, default=4)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
