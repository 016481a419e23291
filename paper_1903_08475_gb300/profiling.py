"""Measurement helpers for the ncu captures behind bench.py's roofline.

    python -m paper_1903_08475_gb300.profiling solves [precision] [n] [n_r]
        runs n config-1 solves (the launches an ncu capture selects from);
    python -m paper_1903_08475_gb300.profiling traffic <ncu.csv> <out.json> [precision] [n_r]
        turns an ncu CSV of dram__bytes_read.sum / dram__bytes_write.sum per
        launch into the per-kernel DRAM bytes bench.py reports, stamped with
        the hash of the CUDA sources the capture ran.

bench.py reports a kernel's traffic only while that hash matches the
sources it runs, so a number never outlives the kernel it was measured on.
"""
from __future__ import annotations

import csv
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "dram_traffic.json")

# phase names bench.py uses, by the kernel-name prefix ncu prints
PHASE_OF_KERNEL = (("tc_gemm_kernel<2, 0", "projection"), ("tc_gemm_kernel<3, 0", "projection"),
                   ("tc_gemm_kernel<1, 0", "projection"),
                   ("tc_gemm_kernel<2, 1", "synthesis"), ("tc_gemm_kernel<3, 1", "synthesis"),
                   ("tc_gemm_kernel<1, 1", "synthesis"),
                   ("field16_kernel", "field_slices"), ("field_slices_kernel", "field_slices"),
                   ("field_slices_tf32_kernel", "field_slices"), ("emu_field_kernel", "field_slices"),
                   ("scan_ff_kernel", "radial_scan"), ("emu_scan_kernel", "radial_scan"),
                   ("slice_m16_kernel", "radial_scan_slices"), ("emu_slice_m_kernel", "radial_scan_slices"))


def sources_sha() -> str:
    """SHA-256 over the library's CUDA sources and internal headers (file
    names and contents, in name order) and the public header."""
    h = hashlib.sha256()
    files = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h")))
    for f in files:
        h.update(f.encode())
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(ROOT, "include", "ygs.h"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def solves(precision: str = "fp16x3", n: int = 2, n_r: int = 400):
    import torch

    from . import Plan, ygs_solve, workloads as W

    grid, rho = W.config1(n_r=n_r)
    with Plan(grid, precision) as plan:
        r = torch.from_numpy(rho).cuda()
        out = torch.empty_like(r)
        for _ in range(n):
            ygs_solve(plan, r, out)
        torch.cuda.synchronize()
    print(f"{n} {precision} solves done")


def _phase(name: str):
    for prefix, phase in PHASE_OF_KERNEL:
        if prefix in name.replace("ygs::tc::", "").replace("ygs::", ""):
            return phase
    return None


def traffic(csv_path: str, out_json: str, precision: str = "fp16x3", n_r: int = 400):
    """Per phase: the median over captured launches of read + write DRAM bytes."""
    per = {}
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f) if r]
    head = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    cols = rows[head]
    ki, mi, vi, ii = cols.index("Kernel Name"), cols.index("Metric Name"), cols.index("Metric Value"), cols.index("ID")
    launches = {}
    for r in rows[head + 1:]:
        if len(r) <= max(ki, mi, vi, ii):
            continue
        key = (r[ii], r[ki])
        try:
            v = float(r[vi].replace(",", ""))
        except ValueError:
            continue
        unit = r[cols.index("Metric Unit")] if "Metric Unit" in cols else "byte"
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}.get(unit, 1)
        if r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            launches.setdefault(key, {})[r[mi]] = v * scale
    for (_, name), m in launches.items():
        phase = _phase(name)
        if phase and len(m) == 2:
            per.setdefault(phase, []).append(m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"])
    out = {"sources_sha256": sources_sha(), "precision": precision, "n_r": n_r,
           "workload": "config 1 (Yin-Yang 1 degree, 92x272x2, Nr 400, l_max 32)",
           "bytes_per_launch": {k: sorted(v)[len(v) // 2] for k, v in per.items()},
           "launches": {k: len(v) for k, v in per.items()},
           "command": ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none "
                       "--csv --log-file traffic.csv python -m paper_1903_08475_gb300.profiling solves "
                       f"{precision} 2 {n_r}")}
    with open(out_json, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    return out


def load_traffic(precision: str, n_r: int, phase: str):
    """DRAM bytes per launch of `phase` from profiles/dram_traffic.json, or
    None when there is none for these sources, precision and workload."""
    try:
        with open(TRAFFIC_JSON) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("sources_sha256") != sources_sha() or t.get("precision") != precision or t.get("n_r") != n_r:
        return None
    v = t.get("bytes_per_launch", {}).get(phase)
    return int(v) if v is not None else None


if __name__ == "__main__":
    cmd = sys.argv[1] if len(sys.argv) > 1 else "solves"
    if cmd == "solves":
        solves(*(sys.argv[2:3] or ["fp16x3"]), *(int(x) for x in sys.argv[3:5]))
    elif cmd == "traffic":
        a = sys.argv[2:]
        print(json.dumps(traffic(a[0], a[1], *(a[2:3]), *(int(x) for x in a[3:4])), indent=1))
    else:
        raise SystemExit(__doc__)
