"""Runs in a child process whose YGS_LIB names the checked build of libygs
(tests/test_gpu_checked_build.py): small solves, adjoints and a batch of
every precision against the CPU FP64 oracle, each followed by
ygs_get_status, which must report no out-of-range index; then, with the
field extent the checks use shrunk by one shell, a solve whose last shell's
accesses the checks must report (and skip).  Prints one line per case and
exits non-zero on the first failure."""
import math
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1903_08475_gb300 import (Batch, Plan, YgsError, ygs_backward, ygs_checked_build,  # noqa: E402
                                    ygs_debug_set_field_extent, ygs_get_status, ygs_solve, workloads as W)

TOL = {"fp64": 1e-12, "fp64emu": 1e-12, "fp16x3": 1e-6, "bf16x6": 1e-6, "bf16x3": 5e-4, "tf32x3": 1e-6,
       "fp32": 1e-4, "fp64tc": 1e-12}


def rel_max(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def main():
    assert ygs_checked_build(), "YGS_LIB does not name the checked build"
    from tests.test_gpu_fp64 import three_patch_grid
    grids = {
        "yy_ragged": W.yinyang_grid(13, 37, math.radians(4.0), W.log_edges(67, 0.05), 9),
        "three_patch": three_patch_grid(),
        "polar": W.polar_grid(7, 13, W.linear_edges(6, 0.1, 1.0), 5),
    }
    for name, grid in grids.items():
        rho = W.random_density(grid, 11)
        ref = oracle.solve(grid, rho)
        g = W.random_density(grid, 12)
        ref_t = oracle.apply_T(grid, g)
        for prec in TOL:
            with Plan(grid, prec) as plan:
                phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
                torch.cuda.synchronize()
                ygs_get_status(plan)
                err = rel_max(phi.cpu().numpy(), ref)
                assert err <= TOL[prec], f"{name} {prec}: {err:.3e}"
                gr = ygs_backward(plan, torch.from_numpy(g).cuda())
                torch.cuda.synchronize()
                ygs_get_status(plan)
                scale = np.abs(ref_t).max()
                err_t = float(np.abs(gr.cpu().numpy() - ref_t).max() / scale)
                assert err_t <= max(10 * TOL[prec], 1e-12), f"{name} {prec} adjoint: {err_t:.3e}"
                print(f"ok {name} {prec} {err:.2e} {err_t:.2e}", flush=True)
    # a batch of uneven fields (grouped launches)
    gb = [W.yinyang_grid(6, 18, math.radians(8.0), W.log_edges(nr, 0.05), lm) for nr, lm in ((9, 6), (20, 4))]
    for prec in ("fp16x3", "bf16x6", "fp64emu"):
        plans = [Plan(x, prec) for x in gb]
        try:
            rhos = [torch.from_numpy(W.random_density(x, 5)).cuda() for x in gb]
            with Batch(plans) as b:
                outs = b.solve(rhos)
            torch.cuda.synchronize()
            for p_, x, r, o in zip(plans, gb, rhos, outs):
                ygs_get_status(p_)
                err = rel_max(o.cpu().numpy(), oracle.solve(x, r.cpu().numpy()))
                assert err <= TOL[prec], f"batch {prec}: {err:.3e}"
        finally:
            for p_ in plans:
                p_.close()
        print(f"ok batch {prec}", flush=True)
    # a check that fires: the extent the checks use one shell short of the field
    grid = grids["yy_ragged"]
    rho = torch.from_numpy(W.random_density(grid, 13)).cuda()
    for prec in ("fp64", "fp16x3", "bf16x6", "fp64emu"):
        with Plan(grid, prec) as plan:
            n = plan.info["n_cells"]
            ygs_debug_set_field_extent(plan, n - plan.info["n_ang"])
            ygs_solve(plan, rho)
            torch.cuda.synchronize()
            try:
                ygs_get_status(plan)
            except YgsError as e:
                assert "YGS_ERR_BOUNDS" in str(e) and "out of range" in str(e), str(e)
                print(f"ok reported {prec}: {e}", flush=True)
            else:
                raise AssertionError(f"{prec}: no out-of-range index reported")
            ygs_debug_set_field_extent(plan, n)
            ygs_solve(plan, rho)
            torch.cuda.synchronize()
            ygs_get_status(plan)  # cleared by the read above, and nothing new
    print("all ok", flush=True)


if __name__ == "__main__":
    main()
