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
FP64_PEAK_TFLOPS = 1.25


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f), "of measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


def _roofline(prec, mode, flops_per_launch, avg_launch_s, launches, n_u=None):
    """Roofline entry of the block matvec (the dominant kernel) for the precision used."""
    achieved = flops_per_launch / avg_launch_s / 1e12
    if prec in ("bf16split", "fp16split"):
        peaks, src = _measured_peaks()
        peak = float(peaks["bf16_tflops_sustained"])
        traffic = None
        if mode == "matfree":
            return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": f"k_tc_mf (tcgen05 {prec} pair kernel: T tiles generated in shared "
                              "memory, 3 MMAs per product)",
                    "peak_source": f"bf16 dense sustained ({src}); algorithmic flops 4 n_u^2 B, "
                                   "executed tensor flops are 3x",
                    "avg_launch_ms": avg_launch_s * 1e3, "launches": launches}
        ratio = _profile_ratio("k_gemm_tc.cu", "k_tc_gemm_fp16split.md")
        if ratio is not None and n_u:
            # algorithmic bytes of the average launch: T hi + lo once, the hi/lo operand
            # and the FP32 result for its 2 B real columns
            np_ = -(-n_u // 128) * 128
            b_avg = flops_per_launch / (4.0 * n_u * n_u)
            traffic = ratio * (4.0 * np_ * np_ + 16.0 * np_ * b_avg)
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": f"k_tc_gemm (tcgen05 {prec} block matvec, 3 MMAs per product)",
                "peak_source": f"bf16 dense sustained ({src}); algorithmic flops 4 n_u^2 B, "
                               "executed tensor flops are 3x",
                "avg_launch_ms": avg_launch_s * 1e3, "launches": launches}
    if prec == "fp64":
        return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "k_dgemm / k_dgemv (FP64 CUDA-core block matvec)",
                "peak_source": "GB300 dense FP64 rate, 1.25 TFLOP/s nominal",
                "avg_launch_ms": avg_launch_s * 1e3, "launches": launches}
    traffic = None
    if mode != "matfree":
        ratio = _profile_ratio("k_gemm_simt.cu", "k_sgemm_fp32.md")
        if ratio is not None and n_u:
            np_ = -(-n_u // 128) * 128
            b_avg = flops_per_launch / (4.0 * n_u * n_u)
            # T (FP32) once, the FP32 operand and result of the 2 B real columns
            traffic = ratio * (4.0 * np_ * np_ + 16.0 * np_ * b_avg)
    return {"bound": "alu", "achieved": achieved, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP32_ALU_PEAK_TFLOPS, "traffic": traffic,
            "kernel": ("k_sgemm_mf (FP32 CUDA-core pair kernel: T tiles generated on the fly)"
                       if mode == "matfree" else
                       "k_sgemm (FP32 CUDA-core block matvec on the materialised T)"),
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz",
            "avg_launch_ms": avg_launch_s * 1e3, "launches": launches}


# Arithmetic the path computes in, per matvec precision: the matvec's operand and
# accumulation types, then the FP64-class (double-FP32 or FP64) true residual and
# refinement.
DTYPES = {"fp16split": "f16-split (3 MMA) / f32 accumulate + f32 basis + f64-class residual",
          "bf16split": "bf16-split (3 MMA) / f32 accumulate + f32 basis + f64-class residual",
          "fp32": "f32 + f32 basis + f64-class residual", "fp64": "f64"}


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
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0=None, t1=None):
        """Median SM clock, its maximum and the throttle reasons of the samples taken in
        [t0, t1] (perf_counter times; all samples when not given or none fall inside)."""
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
        lines = self.lines
        if t0 is not None and t1 is not None:
            inside = [(t, ln) for t, ln in lines if t0 <= t <= t1]
            if inside:
                lines = inside
        for _, ln in lines:
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
                "samples": len(sm),
                "window": "timed region" if lines is not self.lines else "whole run"}


# ---------------------------------------------------------------- roofline traffic
# Device code of a profiled kernel: the text before the file's first host-side launcher
# helper (tensor-core file), or the span from the file's namespace to the next kernel
# (the FP32 GEMM shares its file with the FP64 kernels).  Code outside it does not change
# what the profiled kernel executes.
DEVICE_PART_END = {"k_gemm_tc.cu": b"// Xt_hi[c][k], Xt_lo[c][k] (K-major) from X[k][c]"}
DEVICE_PART_SPAN = {"k_gemm_simt.cu": (b"namespace px {", b"// FP64: BM = BN = 64, BK = 16"),
                    "k_shifted.cu": (b"// ---------------------------------------------------------------- matvec",
                                     b"// U[i][p] = sum over segments")}


def kernel_source_sha(kernel_file):
    """sha256 of the device part of a kernel source (the whole file where no marker is
    listed)."""
    src = os.path.join(ROOT, "paper_2510_12731_gb300", "csrc", kernel_file)
    data = open(src, "rb").read()
    end = DEVICE_PART_END.get(kernel_file)
    if end is not None and end in data:
        data = data[:data.index(end)]
    span = DEVICE_PART_SPAN.get(kernel_file)
    if span is not None and span[0] in data and span[1] in data:
        i = data.index(span[0])
        data = data[i:data.index(span[1], i)]
    return hashlib.sha256(data).hexdigest()


def _profile_ratio(kernel_file, profile_file):
    """Measured DRAM bytes / algorithmic bytes of one captured launch, from a committed
    ncu summary taken on the current device code (None otherwise)."""
    path = os.path.join(ROOT, "profiles", profile_file)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_r = re.search(r"dram_over_algorithmic:\s*([0-9.eE+]+)", text)
    if not (m_sha and m_r) or m_sha.group(1) != kernel_source_sha(kernel_file):
        return None
    return float(m_r.group(1))


# ---------------------------------------------------------------- multi-rank helpers
def max_over_ranks(x, dist=None, device=None):
    """Largest x over all ranks; x itself without an initialised process group."""
    if dist is None or not dist.is_initialized():
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(points_per_step, world, ms_per_step_max):
    """Spectrum points per second of all ranks: every rank (a replica) solves the same
    number of points per step; the job's step takes as long as the slowest rank."""
    return world * points_per_step / (ms_per_step_max / 1e3)


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
    """The FP64 CPU checker on the host cores, on the bench's workload.  One sample is a
    dense LU of the whole system at one frequency for every polarisation (~100 s at
    N = 19,931 on 16 cores), so the timed samples stop once the next one would pass a
    wall-time budget (--ref-budget-s); at least one is always timed, and the line
    reports how many were."""
    if rank != 0:
        return 0
    wl = _workload(args.workload)
    # the untimed warm-up steps run the same code on the 791-atom Ag sphere (BLAS thread
    # pool and allocator warm-up), so they cost seconds, not minutes
    warm_wl = _workload("ag_sphere")
    for _ in range(args.warmup):
        _oracle_sample(warm_wl, 1)
    times = []
    pts = 0
    for _ in range(args.steps):
        dt, p = _oracle_sample(wl, args.cpu_freqs)
        times.append(dt)
        pts = p
        if sum(times) + max(times) > args.ref_budget_s:
            break
    per = sum(times) / len(times)
    value = pts / per
    sample = (f"dense LU (numpy/LAPACK) of the full N={wl.natoms} system for {args.cpu_freqs} "
              f"frequency x {wl.pol_dirs.shape[0]} polarisations per step; {len(times)} of "
              f"{args.steps} requested steps timed within a {args.ref_budget_s:.0f} s budget")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": len(times), "steps_requested": args.steps,
            "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "natoms": wl.natoms, "columns": wl.ncols},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                             "sample": sample},
            "warmup_sample": "dense LU of the 791-atom Ag sphere, 1 frequency",
            "step_s": [round(t, 2) for t in times],
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2510_12731_gb300 import Solver
    if getattr(args, "solver", "batched") == "shifted":
        return run_shifted_main(args, rank, world, local_rank)

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = _workload(args.workload)
    F, P, N = wl.omega_ev.size, wl.pol_dirs.shape[0], wl.natoms
    # profile = 1 times every matvec launch with CUDA events over the timed region (the
    # roofline's kernel duration); restart cycles then run as per-kernel launches.  With
    # --graphs the timed region runs each restart cycle as one graph launch and the
    # kernel duration comes from one profiled step after the timed region.
    opts = dict(precision=args.precision or wl.precision, tol_rel=wl.tol,
                profile=0 if args.graphs else 1, cycle_graphs=1 if args.graphs else 0,
                restart_m=args.restart_m, gs_passes=args.gs_passes, basis=args.basis)
    if args.inner_tol:
        opts["inner_tol"] = args.inner_tol
    opts["mode"] = args.mode or wl.mode
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

    if getattr(args, "profile_run", False):
        return _profile_step(step_device, solver, wl.name, "batched")

    # the clock sampler starts before the warm-up (nvidia-smi's start-up then overlaps the
    # warm-up steps, not the timed ones); only samples inside the timed region are used
    clocks = ClockSampler(local_rank)
    clocks.start()
    for _ in range(args.warmup):
        step_device()
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    mv_ms = 0.0
    mv_n = 0
    mv_flops = 0.0
    converged = 0
    iters = 0
    t_wall0 = time.perf_counter()
    step_wall = []
    ev0.record()
    for _ in range(args.steps):
        ts = time.perf_counter()
        ok = step_device()
        step_wall.append((time.perf_counter() - ts) * 1e3)
        st = solver.stats()
        launches += st["kernel_launches"] + st["setup_launches"]
        mv_ms += st["matvec_ms"]
        mv_n += st["matvec_launches"]
        mv_flops += st["matvec_flops"]
        iters += st["total_iters"]
        # a step that returns ok had every column at or below tol_rel (the library's own
        # FP64-class check); only otherwise are the residuals counted here (a device
        # reduction and a host read, which would otherwise sit inside the timed region)
        converged += F * P if ok else int((d_rr <= wl.tol).sum().item())
    ev1.record()
    torch.cuda.synchronize()
    t_wall1 = time.perf_counter()
    wall = t_wall1 - t_wall0
    clk = clocks.stop(t_wall0, t_wall1)
    ms = ev0.elapsed_time(ev1)
    barrier()
    ms = max_over_ranks(ms, dist, dev)
    points_per_step = converged / args.steps
    value = whole_job_value(points_per_step, world, ms / args.steps)

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
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e_value = whole_job_value(e2e_pts / e2e_steps, world, e2e_ms / e2e_steps)
    h2d = wl.xyz_ang.nbytes + wl.type_idx.nbytes + wl.omega_ev.nbytes + wl.pol_dirs.nbytes + \
        64 * len(wl.types) + (0 if wl.alpha_ib is None else wl.alpha_ib.nbytes)
    d2h = sum(v.nbytes for k, v in out.items() if isinstance(v, np.ndarray)
              and not (k == "sigma_abs" and P != 3))

    # ---- roofline of the dominant kernel (the block matvec)
    prec = opts["precision"]
    kernel_timing = "CUDA events around every matvec launch over the timed region"
    if args.graphs:
        with Solver(**{**opts, "profile": 1, "cycle_graphs": 0}) as ps:
            ps.set_structure(wl.model, wl.xyz_ang, wl.type_idx, wl.types)
            ps.solve_device(wl.omega_ev, wl.pol_dirs, wl.alpha_ib, d_alpha=d_alpha, d_q=d_q,
                            d_relres=d_rr)
            pst = ps.stats()
        mv_ms, mv_n, mv_flops = pst["matvec_ms"], pst["matvec_launches"], pst["matvec_flops"]
        kernel_timing = "CUDA events around every matvec launch of one profiled step after the timed region"
    graph_launches = st["graph_launches"]
    avg_launch_s = (mv_ms / mv_n) / 1e3 if mv_n else float("nan")
    flops_per_launch = mv_flops / mv_n if mv_n else float("nan")
    roofline = _roofline(prec, opts["mode"], flops_per_launch, avg_launch_s, mv_n,
                         n_u=N if wl.model == "wfq" else 4 * N)

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

    shifted = None
    nsk = args.steps if getattr(args, "shifted_steps", 0) < 0 else getattr(args, "shifted_steps", 0)
    if nsk > 0 and wl.model == "wfq":
        shifted = run_shifted_leg(args, wl, nsk, dev, dist, world, d_alpha, d_q, d_rr, pinned,
                                  value)

    # ---- P0, second variant (wFQ, N <= 12,000): one complex LU per frequency of
    # A(w) = Kbar T - z_q(w) I (cuSOLVER through torch) for every direction at once, on
    # the operator the library exports; the faster P0 variant is the denominator
    p0_lu = None
    if args.p0_cols > 0 and wl.model == "wfq" and N <= 12000:
        p0_lu = _p0_lu(wl, dev, args.p0_cols)
    p0_best = p0
    if p0_lu is not None and (p0 is None or p0_lu["value"] > p0["value"]):
        p0_best = p0_lu

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
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES.get(prec, prec),
            "data": "synthetic",
            "config": {"workload": wl.name, "natoms": N, "n_unknowns": N if wl.model == "wfq" else 4 * N,
                       "n_freq": F, "n_pol": P, "columns": F * P, "tol_rel": wl.tol,
                       "precision": prec, "mode": opts["mode"], "restart_m": args.restart_m,
                       "gs_passes": args.gs_passes, "basis": args.basis,
                       "cycle_graphs": bool(args.graphs),
                       "l2": "no flush: the per-step working set (T, Krylov basis) is far larger than L2",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk, "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                                   "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "gpu_launches": launches, "graph_launches_last_step": graph_launches,
            "roofline": {**roofline, "kernel_timing": kernel_timing}, "cpu_baseline": cpu,
            "p0_fp64_gpu": p0, "p0_lu_gpu": p0_lu,
            "vs_p0": (value / world / p0_best["value"]) if p0_best else None,
            "shifted_krylov": shifted,
            "points_per_step": points_per_step, "iters_per_step": iters / args.steps,
            "wall_s": wall, "step_wall_ms": [round(x, 1) for x in step_wall],
        }
        print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def _p0_lu(wl, dev, nsample):
    """Plain FP64 direct solve on the GPU: A(w) = A0 - z_q(w) I assembled in complex128 from
    the library's exported A0 = Kbar T (Eq. 1), one LU with all directions per frequency
    (torch.linalg.solve: cuSOLVER getrf / getrs); timed on sampled frequencies."""
    import torch
    from paper_2510_12731_gb300 import Solver
    N, P = wl.natoms, wl.pol_dirs.shape[0]
    A0 = torch.empty((N, N), dtype=torch.float64, device=dev)
    b = torch.empty((N, P), dtype=torch.float64, device=dev)
    with Solver(precision="fp64", tol_rel=wl.tol) as s:
        s.set_structure(wl.model, wl.xyz_ang, wl.type_idx, wl.types)
        s.system_device(wl.pol_dirs, 1.0, d_A0=A0, d_b=b)
    n, tau = wl.types[0]["drude_n_au"], wl.types[0]["tau_au"]
    bc = b.to(torch.complex128)
    eye = torch.eye(N, dtype=torch.complex128, device=dev)
    fidx = np.unique(np.linspace(0, wl.omega_ev.size - 1, nsample).round().astype(int))

    def solve_one(fi):
        w = wl.omega_ev[fi] / 27.211386245988
        zq = complex(-w * w * tau / (2 * n * tau), -w / (2 * n * tau))   # Eq. 6
        A = A0.to(torch.complex128) - zq * eye
        x = torch.linalg.solve(A, bc)
        rel = (torch.linalg.norm(bc - A @ x, dim=0) / torch.linalg.norm(bc, dim=0)).max()
        return x, rel

    solve_one(fidx[0])                       # library warm-up (cuSOLVER handles, workspace)
    torch.cuda.synchronize()
    t = 0.0
    worst = 0.0
    for fi in fidx:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, rel = solve_one(fi)
        e1.record()
        torch.cuda.synchronize()
        t += e0.elapsed_time(e1) / 1e3
        worst = max(worst, float(rel))
    del A0, eye
    return {"value": len(fidx) * P / t, "unit": UNIT, "frequencies_timed": int(len(fidx)),
            "max_rel_residual": worst,
            "sample": f"{len(fidx)} frequencies x {P} directions, complex128 LU per frequency "
                      "(torch.linalg.solve), A(w) assembled from the exported Kbar T; "
                      "residual check included"}


def _profile_step(step, solver, workload, solver_name):
    """--profile-run: one step of the path, no warm-up and no timing, for launch lists and
    counter captures under a profiler.  Prints a line that carries no bench value."""
    import torch
    step()
    torch.cuda.synchronize()
    st = solver.stats()
    print(json.dumps({"profile_run": True, "workload": workload, "solver": solver_name,
                      "kernel_launches": st["kernel_launches"] + st["setup_launches"],
                      "note": "one untimed step for a profiler; not a bench value"}), flush=True)
    return 0


def run_shifted_leg(args, wl, steps, dev, dist, world, d_alpha, d_q, d_rr, pinned, batched_value):
    """The same workload and step (set-up + solve of every column + observables) with the
    shifted Krylov solver: one real Arnoldi process per field direction for the whole
    sweep (Eq. 1 with the scalar shift of Eq. 6), double-FP32 throughout.  A separate mode,
    reported next to the batched line.  Its dominant kernel, the double-FP32 matvec on the
    directions' columns, streams T's two FP32 planes once per step: HBM-bound."""
    import torch
    from paper_2510_12731_gb300 import Solver
    F, P, N = wl.omega_ev.size, wl.pol_dirs.shape[0], wl.natoms
    # profile = 1 events every shifted matvec (two events per Arnoldi step, ~0.1% of it)
    sk = Solver(solver="shifted", precision="fp32", tol_rel=wl.tol, profile=1)

    def step():
        sk.set_structure(wl.model, wl.xyz_ang, wl.type_idx, wl.types)
        return sk.solve_device(wl.omega_ev, wl.pol_dirs, wl.alpha_ib, d_alpha=d_alpha, d_q=d_q,
                               d_relres=d_rr)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if getattr(args, "profile_run", False):
        return _profile_step(step, sk, wl.name, "shifted")

    for _ in range(max(3, min(args.warmup, 5))):
        step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    conv = 0
    mv_ms = mv_n = mv_bytes = ksteps = launches = 0.0
    e0.record()
    for _ in range(steps):
        ok = step()
        st = sk.stats()
        mv_ms += st["shift_matvec_ms"]
        mv_n += st["shift_matvec_launches"]
        mv_bytes += st["shift_matvec_bytes"]
        ksteps += st["shift_steps"]
        launches += st["kernel_launches"] + st["setup_launches"]
        conv += F * P if ok else int((d_rr <= wl.tol).sum().item())
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    value = whole_job_value(conv / steps, world, ms / steps)
    # end to end: host buffers through px_solve, copies inside the timed region
    xyz_p = pinned(wl.xyz_ang.shape, np.float64)
    xyz_p[...] = wl.xyz_ang
    tid_p = pinned(wl.type_idx.shape, np.int32)
    tid_p[...] = wl.type_idx
    out = sk.alloc_outputs(F, P, want_q=True, want_mu=True, empty=lambda s, dtype: pinned(s, dtype))
    e2e_steps = max(1, min(steps, args.e2e_steps))
    sk.set_structure(wl.model, xyz_p, tid_p, wl.types)
    sk.solve(wl.omega_ev, wl.pol_dirs, wl.alpha_ib, out=out)
    barrier()
    e0.record()
    pts = 0
    for _ in range(e2e_steps):
        sk.set_structure(wl.model, xyz_p, tid_p, wl.types)
        r = sk.solve(wl.omega_ev, wl.pol_dirs, wl.alpha_ib, out=out)
        pts += int((r["status"] == 0).sum())
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    sk.close()
    peaks, src = _measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    avg_s = (mv_ms / mv_n) / 1e3 if mv_n else float("nan")
    achieved = (mv_bytes / mv_n) / avg_s / 1e9 if mv_n else float("nan")
    ratio = _profile_ratio("k_shifted.cu", "k_sk_matvec_na_sphere_7119.md")
    traffic = ratio * (mv_bytes / mv_n) if (ratio is not None and mv_n) else None
    h2d = wl.xyz_ang.nbytes + wl.type_idx.nbytes + wl.omega_ev.nbytes + wl.pol_dirs.nbytes + \
        64 * len(wl.types)
    d2h = sum(v.nbytes for k, v in out.items() if isinstance(v, np.ndarray)
              and not (k == "sigma_abs" and P != 3))
    return {
        "value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
        "points_per_step": conv / steps, "krylov_steps_per_step": ksteps / steps,
        "gpu_launches": int(launches), "vs_batched": value / batched_value if batched_value else None,
        "e2e": {"value": whole_job_value(pts / e2e_steps, world, e2e_ms / e2e_steps), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "kernel": "k_sk_matvec (double-FP32 matvec of T's two FP32 planes on one "
                               "column per field direction)",
                     "peak_source": f"STREAM-style copy ({src})",
                     "algorithmic_bytes_per_launch": mv_bytes / mv_n if mv_n else None,
                     "avg_launch_ms": avg_s * 1e3, "launches": int(mv_n),
                     "kernel_timing": "CUDA events around every shifted matvec over the timed region"},
        "note": "separate mode (Eq. 1: one Krylov space per field direction serves all "
                "frequencies); not part of the batched-vs-P0 comparison"}


def run_shifted_main(args, rank, world, local_rank):
    """The shifted Krylov solver as the line's own measurement (--solver shifted): the same
    step, timed as in the shifted leg, with that leg's roofline, e2e and launch count."""
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = _workload(args.workload)
    if wl.model != "wfq":
        raise SystemExit("--solver shifted applies to wFQ workloads")
    F, P, N = wl.omega_ev.size, wl.pol_dirs.shape[0], wl.natoms
    dev = torch.device("cuda", local_rank)
    d_alpha = torch.empty((F, 3, P), dtype=torch.complex128, device=dev)
    d_q = torch.empty((F, P, N), dtype=torch.complex128, device=dev)
    d_rr = torch.empty((F, P), dtype=torch.float64, device=dev)

    def pinned(shape, dtype):
        t = torch.empty(shape, dtype={np.complex128: torch.complex128, np.float64: torch.float64,
                                      np.int32: torch.int32}[np.dtype(dtype).type], pin_memory=True)
        return t.numpy()

    clocks = ClockSampler(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    sk = run_shifted_leg(args, wl, args.steps, dev, dist, world, d_alpha, d_q, d_rr, pinned, None)
    clk = clocks.stop(t0, time.perf_counter())
    if getattr(args, "profile_run", False):
        return 0
    if rank == 0:
        line = {"metric": METRIC, "value": sk["value"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, min(args.warmup, 5)),
                "ms_per_step": sk["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32-pair (double-FP32) matvec, basis and "
                                              "orthogonalisation + f64 least squares",
                "data": "synthetic",
                "config": {"workload": wl.name, "natoms": N, "n_unknowns": N, "n_freq": F,
                           "n_pol": P, "columns": F * P, "tol_rel": wl.tol, "solver": "shifted",
                           "l2": "no flush: the per-step working set (T planes) is far larger than L2",
                           "parallelism": f"replicas x{world}"},
                "clocks": clk, "e2e": sk["e2e"], "gpu_launches": sk["gpu_launches"],
                "roofline": sk["roofline"], "cpu_baseline": None,
                "points_per_step": sk["points_per_step"],
                "krylov_steps_per_step": sk["krylov_steps_per_step"]}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- boundary elements
def run_bem(args, rank, world, local_rank):
    """Boundary-element sweep (DPCM, Eq. 11, or IEFPCM, Eq. 12, by --bem-formulation): a
    Drude sphere meshed by --bem-tess tesserae,
    200 frequencies x (x, y, z).  One step = px_set_mesh (Ft in FP64 and the solver's
    planes) + px_solve_bem of every column with the results copied to pinned host memory
    (the host-buffer call is the only one: value and e2e coincide except for the tesserae's
    charges, which e2e also copies back).  Shifted solver by default (one Krylov space per
    direction, Lambda(w) as the shift); --solver batched runs the block GMRES."""
    import torch
    from paper_2510_12731_gb300 import Solver
    from paper_2510_12731_gb300 import structures as S
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    wl = S.drude_sphere_mesh(args.bem_tess, nfreq=200)
    F, P, n = wl.omega_ev.size, wl.pol_dirs.shape[0], wl.pos_ang.shape[0]
    prec = args.precision or ("fp32" if args.solver == "shifted" else "bf16split")
    sv = Solver(solver=args.solver, precision=prec, tol_rel=wl.tol, profile=1)

    def pinned(shape, dtype):
        t = torch.empty(shape, dtype={np.complex128: torch.complex128, np.float64: torch.float64,
                                      np.int32: torch.int32}[np.dtype(dtype).type], pin_memory=True)
        return t.numpy()

    sv.set_mesh(wl.pos_ang, wl.normals, wl.area_ang2, wl.radius_ang, args.bem_formulation)
    out_small = sv.alloc_outputs(F, P, want_q=False, want_mu=False, empty=pinned)
    out_full = sv.alloc_outputs(F, P, want_q=True, want_mu=False, empty=pinned)

    def step(out):
        sv.set_mesh(wl.pos_ang, wl.normals, wl.area_ang2, wl.radius_ang, args.bem_formulation)
        return sv.solve_bem(wl.omega_ev, wl.eps2, wl.eps1, wl.pol_dirs, out=out,
                            want_q=out is out_full)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if getattr(args, "profile_run", False):
        return _profile_step(lambda: step(out_small), sv, wl.name, args.solver)

    warm = max(3, min(args.warmup, 5))
    for _ in range(warm):
        step(out_small)
    clocks = ClockSampler(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    pts = 0
    mv_ms = mv_n = mv_bytes = ksteps = launches = 0.0
    mm_ms = mm_n = mm_flops = 0.0
    e0.record()
    for _ in range(args.steps):
        r = step(out_small)
        st = sv.stats()
        pts += int((r["status"] == 0).sum())
        mv_ms += st["shift_matvec_ms"]
        mv_n += st["shift_matvec_launches"]
        mv_bytes += st["shift_matvec_bytes"]
        mm_ms += st["matvec_ms"]
        mm_n += st["matvec_launches"]
        mm_flops += st["matvec_flops"]
        ksteps += st["shift_steps"]
        launches += st["kernel_launches"] + st["setup_launches"]
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier()
    e0.record()
    pts2 = 0
    for _ in range(e2e_steps):
        pts2 += int((step(out_full)["status"] == 0).sum())
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    clk = clocks.stop(t0, time.perf_counter())
    sv.close()
    peaks, src = _measured_peaks()
    if mv_n:
        avg_s = (mv_ms / mv_n) / 1e3
        achieved = (mv_bytes / mv_n) / avg_s / 1e9
        hbm = float(peaks["hbm_gbs"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None,
                "kernel": "k_sk_matvec (double-FP32 matvec of Ft's two FP32 planes)",
                "peak_source": f"STREAM-style copy ({src})",
                "algorithmic_bytes_per_launch": mv_bytes / mv_n, "avg_launch_ms": avg_s * 1e3,
                "launches": int(mv_n)}
    elif mm_n:
        roof = _roofline(prec, "materialised", mm_flops / mm_n, (mm_ms / mm_n) / 1e3, int(mm_n), n)
    else:
        roof = None
    h2d = wl.pos_ang.nbytes + wl.normals.nbytes + wl.area_ang2.nbytes + wl.omega_ev.nbytes + \
        4 * 8 * F + wl.pol_dirs.nbytes
    d2h = sum(v.nbytes for k, v in out_full.items() if isinstance(v, np.ndarray))
    if rank == 0:
        line = {"metric": f"BEM ({args.bem_formulation.upper()}) spectrum points/s", "value": whole_job_value(pts / args.steps, world, ms / args.steps),
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": warm,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None,
                "dtype": (DTYPES.get(prec, prec) if args.solver == "batched"
                          else "f32-pair (double-FP32) matvec, basis and orthogonalisation + f64 least squares"),
                "data": "synthetic",
                "config": {"workload": wl.name, "formulation": args.bem_formulation,
                           "n_tesserae": n, "n_freq": F, "n_pol": P,
                           "columns": F * P, "tol_rel": wl.tol, "solver": args.solver,
                           "precision": prec,
                           "l2": "no flush: the operator planes are far larger than L2",
                           "parallelism": f"replicas x{world}"},
                "clocks": clk, "gpu_launches": int(launches),
                "e2e": {"value": whole_job_value(pts2 / e2e_steps, world, e2e_ms / e2e_steps),
                        "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "steps": e2e_steps},
                "roofline": roof, "cpu_baseline": None,
                "krylov_steps_per_step": ksteps / args.steps,
                "note": "boundary-element model of Sec. 2.3 (Eq. 11), a separate workload"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- serving mix
def run_serving(args, rank, world, local_rank):
    """Continuous batching on a seeded mix: first all requests at once (service
    capacity), then Poisson arrivals at 0.7x that request rate (latency under load)."""
    import torch
    from paper_2510_12731_gb300 import Server
    from paper_2510_12731_gb300 import structures as S

    torch.cuda.set_device(local_rank)
    _, descs = S.serving_mix(n_requests=args.serve_requests, seed=12731, nmin=500,
                             nmax=args.serve_nmax)
    wls = [S.build_request(d) for d in descs]
    prec = args.precision or "fp16split"

    def run(arrivals):
        with Server(max_slots=args.serve_slots, precision=prec, tol_rel=1e-7,
                    solver=args.serve_solver) as srv:
            t0 = time.perf_counter()
            ids = []
            for wl, ta in zip(wls, arrivals):
                dt = ta - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                ids.append(srv.submit(wl.model, wl.xyz_ang, wl.type_idx, wl.types, wl.omega_ev,
                                      wl.pol_dirs, wl.alpha_ib))
            outs = [srv.wait(i, timeout_s=3600) for i in ids]
            wall = time.perf_counter() - t0
            st = srv.stats()
        pts = sum(int((o["rel_residual"] <= 1e-7).sum()) for o in outs)
        return pts, wall, st

    clocks = ClockSampler(local_rank)
    clocks.start()
    pts0, wall0, st0 = run([0.0] * len(wls))
    rate = 0.7 * len(wls) / wall0
    rng = np.random.Generator(np.random.PCG64(12731))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(wls)))
    arrivals -= arrivals[0]
    pts1, wall1, st1 = run(arrivals)
    clk = clocks.stop()
    cols = sum(w.ncols for w in wls)
    line = {"metric": METRIC, "value": pts1 / wall1, "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 0, "ms_per_step": wall1 * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES.get(prec, prec), "data": "synthetic",
            "config": {"workload": "serving_mix", "requests": len(wls), "columns": cols,
                       "natoms_range": [min(w.natoms for w in wls), max(w.natoms for w in wls)],
                       "wfqfmu_requests": sum(w.model == "wfqfmu" for w in wls),
                       "slots": args.serve_slots, "precision": prec,
                       "wfq_solver": args.serve_solver,
                       "arrivals": f"Poisson, rate 0.7 x measured capacity = {rate:.3f} req/s"},
            "clocks": clk,
            "serving": {"capacity_points_per_s": pts0 / wall0, "capacity_wall_s": wall0,
                        "points": pts1, "p50_latency_ms": st1["p50_latency_ms"],
                        "p99_latency_ms": st1["p99_latency_ms"],
                        "max_latency_ms": st1["max_latency_ms"],
                        "structure_reuses": st1["structure_reuses"],
                        "peak_reserved_gb": st1["peak_reserved_bytes"] / 1e9,
                        "saturated_p50_ms": st0["p50_latency_ms"],
                        "saturated_p99_ms": st0["p99_latency_ms"]}}
    print(json.dumps(line), flush=True)
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
    ap.add_argument("--restart-m", dest="restart_m", type=int, default=0)
    ap.add_argument("--gs-passes", dest="gs_passes", type=int, default=1)
    ap.add_argument("--basis", default="auto", choices=["auto", "fp64", "ff32", "fp32"])
    ap.add_argument("--graphs", action=argparse.BooleanOptionalAction, default=True,
                    help="run restart cycles as graph launches in the timed region (default; "
                         "--no-graphs: one launch per kernel, every matvec event-timed)")
    ap.add_argument("--solver", default="batched", choices=["batched", "shifted"],
                    help="solver of the main line (the batched line also reports a shifted leg)")
    ap.add_argument("--shifted-steps", dest="shifted_steps", type=int, default=-1,
                    help="timed steps of the shifted Krylov leg (wFQ workloads; -1 = --steps, "
                         "0 = skip)")
    ap.add_argument("--inner-tol", dest="inner_tol", type=float, default=None)
    ap.add_argument("--e2e-steps", dest="e2e_steps", type=int, default=2)
    ap.add_argument("--cpu-freqs", dest="cpu_freqs", type=int, default=1)
    ap.add_argument("--ref-budget-s", dest="ref_budget_s", type=float, default=240.0,
                    help="wall-time budget of the reference arm's timed samples")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--p0-cols", dest="p0_cols", type=int, default=4)
    ap.add_argument("--serve-requests", dest="serve_requests", type=int, default=40)
    ap.add_argument("--serve-nmax", dest="serve_nmax", type=int, default=8000)
    ap.add_argument("--serve-slots", dest="serve_slots", type=int, default=4)
    ap.add_argument("--serve-solver", dest="serve_solver", default="shifted",
                    choices=["batched", "shifted"],
                    help="solver of the served wFQ requests (wFQFmu requests are batched)")
    ap.add_argument("--profile-run", dest="profile_run", action="store_true",
                    help="run one untimed step of the selected path and exit (for profilers)")
    ap.add_argument("--bem-formulation", dest="bem_formulation", default="dpcm",
                    choices=["dpcm", "iefpcm"], help="boundary-element formulation (Eq. 11 or 12)")
    ap.add_argument("--bem-tess", dest="bem_tess", type=int, default=20000,
                    help="tesserae of the boundary-element workload (--workload bem_sphere)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "serving":
        return run_serving(args, rank, world, local_rank)
    if args.workload == "bem_sphere":
        return run_bem(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
