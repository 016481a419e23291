"""Benchmark: Phi solves/s and Gcell/s on the Yin-Yang 1 degree grid
(92 x 272 cells per patch, Nr = 400 log-spaced shells in [1e-3, 1], l_max = 32),
density = rotated tri-axial ellipsoid + 3 Gaussian blobs (seeded, synthetic).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--impl ygs|reference]

One JSON line on rank 0.  `value` is whole-job solves/s over the timed region
(CUDA events on the solve stream, max over ranks, inputs resident in HBM);
`e2e` is the same metric through ygs_solve_host_many (pinned host buffers,
every step's host<->device copies inside the timed region, overlapped with the
neighbouring steps' solves; the one-step-per-call ygs_solve_host figure is
reported beside it); `roofline` is the dominant
kernel's achieved rate against the measured peak; `cpu_baseline` is the CPU
FP64 oracle timed on a bounded sample of the same workload.  With
`--impl reference` the oracle itself is the timed arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Φ solves/s & Gcell/s at l_max; split-prec vs FP64 GPU at ≤1e-6 rel err; % roofline"


def workload_name(n_r: int) -> str:
    return f"yinyang-1deg-92x272x2-Nr{n_r}-lmax32-ellipsoid+3blobs"
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # derived from the SM count, FP32 lanes and max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ygs", choices=["ygs", "reference"])
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-config2", action="store_true",
                    help="skip the config-2 leg (0.5 degree, Nr 800, l_max 64) of the default run")
    ap.add_argument("--n-r", type=int, default=400)
    ap.add_argument("--autotune", action="store_true",
                    help="plans pick their split-K count by timing candidates at create")
    ap.add_argument("--workload", default="config1", choices=["config1", "config2", "config3", "config4"],
                    help="config1: the 1-degree Yin-Yang field (default); config2: 0.5 degree, Nr 800, "
                         "l_max 64, split precision against the FP64 tensor-core path; "
                         "config3: a batch of 64 uneven fields; config4: forward + adjoint, 1 degree, Nr 256")
    return ap.parse_args()


def dist_env():
    from paper_1903_08475_gb300 import dist
    return dist.env()


def measure_fp64_peak(dev) -> float:
    """FP64 TFLOP/s of a cuBLAS DGEMM (torch.matmul, 4096^3, best of 5 after a
    warm-up; CUDA events), the same kind of measurement as the driver's BF16
    peak: the denominator of the FP64 paths' roofline."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ygs_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_sample(grid, rho, n_shells=40):
    """Times the FP64 oracle (weights prebuilt) on `n_shells` of the grid's
    shells with the full angular grid; returns solves/s scaled to all shells."""
    import numpy as np

    import oracle
    from paper_1903_08475_gb300 import workloads as W

    lo = grid.n_r // 2 - n_shells // 2
    sub = W.Grid(**{**grid.__dict__, "edges": grid.edges[lo: lo + n_shells + 1]})
    parts = []
    for p in range(grid.n_patch):
        off, na = grid.patch_offset(p), grid.nang(p)
        parts.append(rho[off + lo * na: off + (lo + n_shells) * na])
    rho_s = np.concatenate(parts)
    U = oracle.build_U(sub)
    Q = oracle.build_Q(sub)
    t0 = time.perf_counter()
    oracle.solve_prebuilt(sub, U, Q, rho_s)
    dt = time.perf_counter() - t0
    full = dt * grid.n_r / n_shells
    return {"value": 1.0 / full, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n_shells} of {grid.n_r} shells (full angular grid, weights prebuilt), "
                      f"{dt:.2f} s, scaled by {grid.n_r}/{n_shells}"}


def run_reference(args, ws, rank):
    """The CPU FP64 oracle as the timed arm (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1903_08475_gb300 import workloads as W

    grid, rho = W.config1(n_r=args.n_r)
    # shells per step: ~4.5 ms of 16-core oracle time per shell plus ~9 ms per call (streaming
    # U and Q once), sized so the whole run stays near two and a half minutes; more shells per
    # call amortise the fixed part (16 shells at the default 2000 + 20 steps)
    n_shells = max(1, min(40, int(150.0 / (max(1, args.steps + args.warmup) * 0.0045))))
    lo = grid.n_r // 2 - n_shells // 2
    sub = W.Grid(**{**grid.__dict__, "edges": grid.edges[lo: lo + n_shells + 1]})
    rho_s = np.concatenate([rho[grid.patch_offset(p) + lo * grid.nang(p): grid.patch_offset(p) + (lo + n_shells) * grid.nang(p)]
                            for p in range(grid.n_patch)])
    U = oracle.build_U(sub)
    Q = oracle.build_Q(sub)
    for _ in range(args.warmup):
        oracle.solve_prebuilt(sub, U, Q, rho_s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve_prebuilt(sub, U, Q, rho_s)
    dt = (time.perf_counter() - t0) / args.steps * grid.n_r / n_shells
    value = 1.0 / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "gcell_per_s": value * grid.n_cells / 1e9,
            "config": {"workload": workload_name(grid.n_r), "n_r": grid.n_r, "l_max": grid.l_max, "cells": grid.n_cells,
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{n_shells} of {grid.n_r} shells per step, weights prebuilt, scaled"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_config3(args, ws, rank, local):
    """64 uneven fields (config 3): the grouped persistent batch replayed from a
    CUDA graph against per-field launches; fields/s over K steps of the whole
    batch, every field resident in HBM (1.0e9 cells, inputs far above L2)."""
    import torch

    from paper_1903_08475_gb300 import Batch, Plan, ygs_launches_per_solve, ygs_solve, workloads as W
    from paper_1903_08475_gb300 import dist as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    precision = args.precision or "fp16x3"
    fields = W.config3()
    plans = [Plan(g, precision, device=local, autotune=args.autotune) for g, _, _ in fields]
    rhos = [W.batch_density(g, kind, seed, device=dev) for g, kind, seed in fields]
    cells = sum(g.n_cells for g, _, _ in fields)
    stream = torch.cuda.Stream(device=dev)
    ref = [torch.empty_like(r) for r in rhos]
    out = [torch.empty_like(r) for r in rhos]

    def per_field():
        for p, r, o in zip(plans, rhos, ref):
            ygs_solve(p, r, o, stream=stream)

    batch = Batch(plans)
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            per_field()
            batch.solve(rhos, out, stream=stream)
    stream.synchronize()
    identical = all(torch.equal(a, b) for a, b in zip(ref, out))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        batch.solve(rhos, out, stream=stream)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                fn()
        e1.record(stream)
        stream.synchronize()
        return D.max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms_graph = timed(graph.replay)
    clk = clocks.stop()
    ms_each = timed(per_field)
    n = len(fields)
    line = {"metric": "fields/s on a batch of 64 uneven fields (config 3)", "value": ws * n / (ms_graph / 1e3),
            "unit": "fields/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": precision,
            "data": "synthetic", "gcell_per_s": ws * cells / (ms_graph / 1e3) / 1e9,
            "config": {"workload": "batch64-uneven-Nr128..600-deg2/1.5/1-lmax16..48-yinyang/6patch",
                       "fields": n, "cells": cells, "precision": precision,
                       "l2": "inputs larger than L2 (1.0e9 cells)", "parallelism": f"replicas{ws}"},
            "per_field_launches": {"fields_per_s": ws * n / (ms_each / 1e3), "ms_per_step": ms_each,
                                   "launches_per_step": sum(ygs_launches_per_solve(p) for p in plans)},
            "speedup_vs_per_field": ms_each / ms_graph, "bitwise_equal_to_per_field": identical,
            "gpu_launches": args.steps * batch.launches, "clocks": clk}
    if args.autotune:
        # the shapes the plans' autotuners kept: (synthesis shells per tile, CTA pairs, split-K) -> plans
        from collections import Counter
        kept = Counter((p.info["synth_tile_shells"], p.info["cta_pairs"], p.info["split_k"]) for p in plans)
        line["config"]["autotune"] = True
        line["autotuned_shapes"] = {f"w{w}-pairs{c}-splitk{k}": v for (w, c, k), v in sorted(kept.items())}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    for p in plans:
        p.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def config2_leg(precision, steps, warmup, local, fp64_cuda_core=True):
    """0.5-degree Yin-Yang, Nr = 800, l_max = 64 (1.6e8 cells, 4225 columns): the
    split path timed against the FP64 tensor-core (and FP64 CUDA-core) paths on
    the same field, with the error of Phi and of B and M per degree band
    (relative 2-norm of each degree's columns).  Returns a dict."""
    import torch

    from paper_1903_08475_gb300 import Plan, ygs_get_moments, ygs_solve, workloads as W
    from paper_1903_08475_gb300 import dist as D

    dev = torch.device("cuda", local)
    grid = W.config2_grid()
    rho = W.lognormal_density_torch(grid, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def timed(plan, n, out, warm):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                ygs_solve(plan, rho, out, stream=stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(n):
                ygs_solve(plan, rho, out, stream=stream)
        e1.record(stream)
        stream.synchronize()
        return D.max_over_ranks(e0.elapsed_time(e1) / n, dev)

    res, outs, moments = {}, {}, {}
    clocks = ClockSampler(local)
    clk = None
    legs = [(precision, steps), ("fp64tc", 1)] + ([("fp64", 1)] if fp64_cuda_core else []) + (
        [("fp64emu", 2)] if precision != "fp64emu" else [])
    for prec, n in legs:
        with Plan(grid, prec, device=local) as plan:
            out = torch.empty_like(rho)
            if prec == precision:
                clocks.start()
                time.sleep(0.3)
            res[prec] = timed(plan, n, out, max(1, min(3, warmup)) if prec == precision else 1)
            if prec == precision:
                clk = clocks.stop()
            ygs_solve(plan, rho, out, stream=stream)
            B, M = ygs_get_moments(plan, stream=stream)
            stream.synchronize()
            outs[prec], moments[prec] = out, (B, M)
    ref, got = outs["fp64tc"], outs[precision]
    rel = float(((got - ref).abs() / ref.abs()).max().item())

    def bands(X, Y):
        errs = []
        for l in range(grid.l_max + 1):
            a, b = X[:, l * l:(l + 1) ** 2], Y[:, l * l:(l + 1) ** 2]
            errs.append(float(torch.linalg.norm(a - b) / max(float(torch.linalg.norm(b)), 1e-300)))
        return errs

    eB = bands(moments[precision][0], moments["fp64tc"][0])
    eM = bands(moments[precision][1], moments["fp64tc"][1])
    ms = res[precision]
    out = {"workload": "yinyang-0.5deg-184x544x2-Nr800-lmax64-lognormal", "cells": grid.n_cells, "K": grid.K,
           "precision": precision, "steps": steps, "ms_per_step": ms, "solves_per_s": 1e3 / ms,
           "gcell_per_s": grid.n_cells / (ms / 1e3) / 1e9,
           "fp64_tensor_solves_per_s": 1e3 / res["fp64tc"], "speedup_vs_fp64_tensor": res["fp64tc"] / ms,
           "max_rel_err_phi_vs_fp64_tensor": rel,
           "B_rel_err_per_l_band": {l: eB[l] for l in range(0, grid.l_max + 1, 8)},
           "M_rel_err_per_l_band": {l: eM[l] for l in range(0, grid.l_max + 1, 8)},
           "B_rel_err_max_over_l": max(eB), "M_rel_err_max_over_l": max(eM), "clocks": clk}
    if "fp64emu" in res and precision != "fp64emu":
        # the FP64-accurate split against the FP64 tensor cores on the same field
        ge = outs["fp64emu"]
        out["fp64emu"] = {"solves_per_s": 1e3 / res["fp64emu"], "speedup_vs_fp64_tensor": res["fp64tc"] / res["fp64emu"],
                          "max_rel_err_phi_vs_fp64_tensor": float(((ge - ref).abs() / ref.abs()).max().item()),
                          "B_rel_err_max_over_l": max(bands(moments["fp64emu"][0], moments["fp64tc"][0])),
                          "M_rel_err_max_over_l": max(bands(moments["fp64emu"][1], moments["fp64tc"][1]))}
    if "fp64" in res:
        out["fp64_cuda_core_solves_per_s"] = 1e3 / res["fp64"]
        out["fp64_tensor_equals_cuda_core_bitwise"] = bool(torch.equal(outs["fp64"], outs["fp64tc"]))
    del outs, moments, rho
    torch.cuda.empty_cache()
    return out


def run_config2(args, ws, rank, local):
    """Config 2 on its own line (``--workload config2``)."""
    import torch

    torch.cuda.set_device(local)
    precision = args.precision or "fp16x3"
    c2 = config2_leg(precision, args.steps, args.warmup, local)
    ms = c2["ms_per_step"]
    line = {"metric": "Phi solves/s, 0.5-degree Yin-Yang Nr 800 l_max 64 (config 2)", "value": ws * 1e3 / ms,
            "unit": "solves/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": precision,
            "data": "synthetic", "gcell_per_s": ws * c2["gcell_per_s"],
            "config": {"workload": c2["workload"], "cells": c2["cells"], "K": c2["K"], "precision": precision,
                       "l2": "inputs larger than L2 (rho 1.3 GB)"},
            **{k: v for k, v in c2.items() if k not in ("workload", "cells", "K", "precision", "steps", "ms_per_step")}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_config4(args, ws, rank, local):
    """The adjoint workload (1 degree Yin-Yang, Nr = 256, l_max = 32, w ~ N(0, 1)):
    one step = Phi = A rho and grad = A^T w (what a gradient of J = sum w Phi
    costs), split precision against the FP64 adjoint."""
    import torch

    from paper_1903_08475_gb300 import Plan, ygs_backward, ygs_solve, workloads as W
    from paper_1903_08475_gb300 import dist as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    precision = args.precision or "fp16x3"
    grid, rho_h, w_h = W.config4()
    rho = torch.from_numpy(rho_h).to(dev)
    w = torch.from_numpy(w_h).to(dev)
    stream = torch.cuda.Stream(device=dev)

    def run(plan, steps):
        phi, g = torch.empty_like(rho), torch.empty_like(rho)
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                ygs_solve(plan, rho, phi, stream=stream)
                ygs_backward(plan, w, g, stream=stream)
        stream.synchronize()
        t = []
        for part in ("both", "backward"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            with torch.cuda.stream(stream):
                for _ in range(steps):
                    if part == "both":
                        ygs_solve(plan, rho, phi, stream=stream)
                    ygs_backward(plan, w, g, stream=stream)
            e1.record(stream)
            stream.synchronize()
            t.append(D.max_over_ranks(e0.elapsed_time(e1) / steps, dev))
        return t, phi, g

    clocks = ClockSampler(local)
    with Plan(grid, precision, device=local) as plan:
        clocks.start()
        time.sleep(0.3)
        (ms_both, ms_bwd), phi, g = run(plan, args.steps)
        clk = clocks.stop()
    with Plan(grid, "fp64", device=local) as p64:
        (ms64, ms64_bwd), phi64, g64 = run(p64, 2)
    rel_g = float(((g - g64).abs().max() / g64.abs().max()).item())
    dot = abs(float((w * phi).sum()) - float((g * rho).sum())) / float((w.abs() * phi.abs()).sum())
    line = {"metric": "forward + adjoint steps/s, 1 degree Yin-Yang Nr 256 l_max 32 (config 4)",
            "value": ws * 1e3 / ms_both, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_both, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": precision, "data": "synthetic",
            "config": {"workload": "yinyang-1deg-92x272x2-Nr256-lmax32-adjoint-w~N(0,1)", "cells": grid.n_cells,
                       "precision": precision},
            "backward_ms": ms_bwd, "fp64_step_ms": ms64, "fp64_backward_ms": ms64_bwd,
            "speedup_vs_fp64": ms64 / ms_both, "adjoint_max_err_vs_fp64_rel_to_max": rel_g,
            "dot_product_identity_residual": dot, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "config3":
        run_config3(args, ws, rank, local)
        return
    if args.workload == "config2":
        run_config2(args, ws, rank, local)
        return
    if args.workload == "config4":
        run_config4(args, ws, rank, local)
        return

    import numpy as np
    import torch

    from paper_1903_08475_gb300 import (Plan, ygs_launches_per_solve, ygs_read_phase_times, ygs_set_profiling,
                                        ygs_solve, ygs_solve_host, ygs_solve_host_many, workloads as W)
    from paper_1903_08475_gb300 import dist as D

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    precision = args.precision or "fp16x3"
    grid, rho = W.config1(n_r=args.n_r)
    plan = Plan(grid, precision, device=local, autotune=args.autotune)
    stream = torch.cuda.Stream(device=dev)
    rho_d = torch.from_numpy(rho).to(dev)
    phi_d = torch.empty_like(rho_d)
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            ygs_solve(plan, rho_d, phi_d, stream=stream)
    stream.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    clocks = ClockSampler(local)
    ygs_set_profiling(plan, True)
    ygs_read_phase_times(plan)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        ygs_solve(plan, rho_d, phi_d, stream=stream)
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    phase_ms, ncalls = ygs_read_phase_times(plan)
    ygs_set_profiling(plan, False)
    ms = D.max_over_ranks(ms, dev)  # the job's time is the slowest rank's
    ms_step = ms / args.steps
    value = ws / (ms_step / 1e3)

    # end to end through the host-buffer entry points: every step copies its
    # field in from pinned host memory and its Phi back.  ygs_solve_host_many
    # overlaps step k's solve with the copies of steps k + 1 and k - 1 (the
    # timed number); ygs_solve_host does one step at a time (reported beside it)
    h_rho = [torch.from_numpy(rho).pin_memory(), torch.from_numpy(rho * 1.5).pin_memory()]
    h_phi = [torch.empty_like(h_rho[0]).pin_memory() for _ in range(2)]
    n_e2e = max(3, min(args.steps, 20))
    many_in = [h_rho[k % 2] for k in range(n_e2e)]
    many_out = [h_phi[k % 2] for k in range(n_e2e)]
    ygs_solve_host_many(plan, many_in[:2], many_out[:2], stream=stream)
    barrier()
    t0 = time.perf_counter()
    ygs_solve_host_many(plan, many_in, many_out, stream=stream)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_s = D.max_over_ranks(e2e_s, dev)
    ygs_solve_host(plan, h_rho[0], h_phi[0], stream=stream)
    n_single = max(3, min(args.steps, 10))
    barrier()
    t0 = time.perf_counter()
    for _ in range(n_single):
        ygs_solve_host(plan, h_rho[0], h_phi[0], stream=stream)
    e2e_single_s = D.max_over_ranks((time.perf_counter() - t0) / n_single, dev)

    # roofline of the dominant kernel
    from paper_1903_08475_gb300.profiling import load_traffic
    peaks, peak_src = load_peaks()
    info = plan.info
    sym = info["symmetric"] == 1
    nang_eff = grid.nang(0) if sym else grid.nang_total
    nprod = {"fp64": 1, "fp64tc": 1, "fp32": 1, "bf16x3": 3, "bf16x6": 6, "fp16x3": 3, "tf32x3": 3,
             "fp64emu": 26}[precision]
    # algorithmic FLOPs of one contraction: one FMA per (shell, stored cell, column) and slice product
    flops_gemm = 2.0 * nprod * grid.n_r * nang_eff * grid.K
    per = [x / max(ncalls, 1) for x in phase_ms]
    names = ["field_slices", "projection", "radial_scan", "synthesis"]
    dom = int(np.argmax(per))
    if precision in ("fp64", "fp64tc", "fp32"):
        flops = [0.0, flops_gemm, 0.0, flops_gemm][dom]
        achieved = flops / (per[dom] / 1e3) / 1e12
        if precision == "fp32":
            pk = NOMINAL_FP32_TFLOPS
            src = "FP32 lanes: 152 SMs x 128 x 2 FLOP x 2.07 GHz (recipe's unit counts and clock)"
        else:
            pk = measure_fp64_peak(dev)
            src = "cuBLAS DGEMM 4096^3 measured in this run (torch.matmul, best of 5)"
        roof = {"kernel": names[dom], "bound": "alu", "achieved": achieved, "peak": pk,
                "unit": "TFLOP/s", "frac": achieved / pk, "traffic": None, "peak_source": src,
                "phase_ms": dict(zip(names, per))}
    else:
        if dom in (1, 3):
            achieved = flops_gemm / (per[dom] / 1e3) / 1e12
            # TF32 runs at half the BF16 dense rate (nominal 1.1 vs 2.25 PFLOP/s)
            peak = float(peaks["bf16_tflops"]) * (1.1 / 2.25 if precision == "tf32x3" else 1.0)
            roof = {"kernel": names[dom], "bound": "tensor", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": load_traffic(precision, grid.n_r, names[dom]),
                    "peak_source": f"bf16_tflops ({peak_src}, burst)" + (
                        "; FP16 dense rate = BF16's (nominal ratio 1)" if precision == "fp16x3" else "") + (
                        "; x 1.1/2.25, the nominal TF32:BF16 ratio" if precision == "tf32x3" else ""),
                    "phase_ms": dict(zip(names, per))}
        else:
            # bytes of the field pass: rho in (FP64) + slices out
            nsl = 3 if precision == "bf16x6" else 2
            byts = grid.n_cells * 8 + grid.n_cells * 2 * nsl
            achieved = byts / (per[dom] / 1e3) / 1e9
            peak = float(peaks["hbm_gbs"])
            roof = {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "traffic": load_traffic(precision, grid.n_r, names[dom]), "peak_source": f"hbm_gbs ({peak_src})",
                    "phase_ms": dict(zip(names, per))}

    # the plain FP64 GPU path on the same input: speed-up and accuracy of the split path against it
    extra = {}
    if precision != "fp64" and not args.no_fp64_compare:
        with Plan(grid, "fp64", device=local) as p64:
            phi64 = torch.empty_like(rho_d)
            ygs_solve(p64, rho_d, phi64, stream=stream)
            stream.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(2):
                ygs_solve(p64, rho_d, phi64, stream=stream)
            f1.record(stream)
            stream.synchronize()
            ms64 = f0.elapsed_time(f1) / 2
            ygs_solve(plan, rho_d, phi_d, stream=stream)
            stream.synchronize()
            rel = float(((phi_d - phi64).abs() / phi64.abs()).max().item())
        extra = {"fp64_gpu_solves_per_s": 1e3 / ms64, "speedup_vs_fp64_gpu": ms64 / ms_step,
                 "max_rel_err_vs_fp64_gpu": rel}
        # the FP64-accurate split (YGS_FP64_EMU) on the same field: its rate,
        # its speed-up over the FP64 CUDA-core path and its error against it
        if precision != "fp64emu":
            try:
                with Plan(grid, "fp64emu", device=local) as pe:
                    phie = torch.empty_like(rho_d)
                    for _ in range(2):
                        ygs_solve(pe, rho_d, phie, stream=stream)
                    stream.synchronize()
                    n_emu = max(3, min(args.steps, 10))
                    f0.record(stream)
                    for _ in range(n_emu):
                        ygs_solve(pe, rho_d, phie, stream=stream)
                    f1.record(stream)
                    stream.synchronize()
                    ms_e = f0.elapsed_time(f1) / n_emu
                    rel_e = float(((phie - phi64).abs() / phi64.abs()).max().item())
                extra["fp64emu"] = {"solves_per_s": 1e3 / ms_e, "ms_per_solve": ms_e,
                                    "gcell_per_s": grid.n_cells / (ms_e / 1e3) / 1e9,
                                    "speedup_vs_fp64_gpu": ms64 / ms_e, "max_rel_err_vs_fp64_gpu": rel_e,
                                    "steps": n_emu}
            except Exception as e:  # context; never lose the headline line over it
                extra["fp64emu"] = {"error": repr(e)}

    # the largest single-GPU configuration beside it (config 2: 0.5 degree,
    # Nr 800, l_max 64), a short leg of the same precision
    if not args.no_config2:
        try:
            extra["config2"] = config2_leg(precision, max(3, min(20, args.steps)), args.warmup, local,
                                           fp64_cuda_core=False)
        except Exception as e:  # context; never lose the headline line over it
            extra["config2"] = {"error": repr(e)}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp64tc": "f64", "fp32": "f32", "fp64emu": "bf16x26 (fp64-accurate)"}.get(precision, precision), "data": "synthetic",
            "gcell_per_s": value * grid.n_cells / 1e9,
            "config": {"workload": workload_name(grid.n_r), "precision": precision, "n_r": grid.n_r, "l_max": grid.l_max,
                       "cells": grid.n_cells, "symmetric": sym, "split_k": info["split_k"], "autotune": args.autotune,
                       "synth_tile_shells": info.get("synth_tile_shells"), "cta_pairs": info.get("cta_pairs"),
                       "l2": "inputs larger than L2 (rho 160 MB, weights 436 MB)",
                       "parallelism": f"replicas{ws}"},
            "e2e": {"value": ws / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": int(rho.nbytes),
                    "d2h_bytes_per_step": int(rho.nbytes), "api": f"ygs_solve_host_many ({n_e2e} steps, copies overlapped)",
                    "single_call": {"value": ws / e2e_single_s, "api": "ygs_solve_host (one step per call)"}},
            "gpu_launches": args.steps * ygs_launches_per_solve(plan),
            "roofline": roof, "clocks": clk, "peaks_source": peak_src, **extra}
    if rank == 0 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline_sample(grid, rho)
        except Exception as e:  # the baseline is context; never lose the GPU line over it
            line["cpu_baseline"] = {"error": repr(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
