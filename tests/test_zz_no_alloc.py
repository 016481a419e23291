"""ygs_solve_static (FP64 solve on a file-scope device scratch array, no device
allocation inside the call) against ygs_solve, through the C ABI.  Kept in a
file collected last so that it also runs after every other GPU test has used
the library in the same process; each case also holds when the file runs
alone in a fresh process."""
import math

import numpy as np
import pytest

from paper_1903_08475_gb300 import (Plan, YgsError, ygs_solve, ygs_solve_static, ygs_static_scratch_capacity,
                                    workloads as W)
from tests._util import rel_max, small_yinyang

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def _need(info):
    return (info["fp64_split_k"] + 2) * info["n_r"] * info["K"] * 8


def _grids():
    return {
        "yy_small": small_yinyang(W),
        "yy_ragged": small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9),
        "yy_1deg_nr100_lmax32": W.yinyang_grid(92, 272, math.radians(1.0), W.log_edges(100, 1e-3, 1.0), 32),
    }


@pytest.mark.parametrize("name", ["yy_small", "yy_ragged", "yy_1deg_nr100_lmax32"])
def test_static_matches_solve_twice(name, cuda):
    """Two calls in a row match ygs_solve; the first call after a fresh
    ygs_create already takes no device memory (the plan loaded the array)."""
    import torch
    grid = _grids()[name]
    rho = torch.from_numpy(W.random_density(grid, 11)).to(cuda)
    phi1 = torch.empty_like(rho)
    phi2 = torch.full_like(rho, float("nan"))
    with Plan(grid, "fp64") as plan:
        assert plan.info["static_scratch_bytes"] == _need(plan.info) <= ygs_static_scratch_capacity()
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ygs_solve_static(plan, rho, phi1)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        ygs_solve_static(plan, rho, phi2)
        torch.cuda.synchronize()
        free2 = torch.cuda.mem_get_info()[0]
        ref = ygs_solve(plan, rho)
        ref, phi1, phi2 = ref.cpu().numpy(), phi1.cpu().numpy(), phi2.cpu().numpy()
    assert rel_max(phi1, ref) <= FP64_TOL
    assert rel_max(phi2, ref) <= FP64_TOL
    assert free1 >= free0 and free2 >= free1  # neither call took device memory


def test_static_on_split_precision_plan_is_fp64(cuda):
    """On a BF16x6 plan the static solve still runs the FP64 kernels on the
    plan's FP64 weights, so it matches the FP64 plan's solve; its scratch is
    sized by the FP64 chunk count, which the info reports beside split_k."""
    import torch
    grid = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    rho = torch.from_numpy(W.random_density(grid, 12)).to(cuda)
    with Plan(grid, "fp64") as p64, Plan(grid, "bf16x6") as p6:
        assert p6.info["static_scratch_bytes"] == _need(p6.info)
        assert p6.info["fp64_split_k"] == p64.info["split_k"]
        ref = ygs_solve(p64, rho).cpu().numpy()
        out = [ygs_solve_static(p6, rho, torch.empty_like(rho)).cpu().numpy() for _ in range(2)]
    for o in out:
        assert rel_max(o, ref) <= FP64_TOL


def test_static_at_and_past_the_limit(cuda):
    """A plan whose scratch is exactly the capacity solves; one shell more is
    rejected with its size in the message, and nothing is enqueued.  Two small
    patches without the Yin-Yang symmetry keep one FP64 chunk each, so the
    need is (2 + 2) n_r K doubles: n_r = 1024, l_max = 31 (K = 1024) gives
    exactly 32 MiB."""
    import torch
    cap = ygs_static_scratch_capacity()
    for n_r, fits in ((1024, True), (1025, False)):
        grid = small_yinyang(W, n_r=n_r, l_max=31)
        with Plan(grid, "fp64", symmetry=False) as plan:
            need = plan.info["static_scratch_bytes"]
            assert need == _need(plan.info)
            rho = torch.from_numpy(W.random_density(grid, 13)).to(cuda)
            phi = torch.zeros_like(rho)
            if fits:
                assert need == cap, "the grid was chosen to need exactly the capacity"
                ygs_solve_static(plan, rho, phi)
                ref = ygs_solve(plan, rho)
                torch.cuda.synchronize()
                assert rel_max(phi.cpu().numpy(), ref.cpu().numpy()) <= FP64_TOL
            else:
                assert need > cap
                with pytest.raises(YgsError) as e:
                    ygs_solve_static(plan, rho, phi)
                assert "UNSUPPORTED" in str(e.value) and str(need) in str(e.value)
                torch.cuda.synchronize()
                assert float(phi.abs().max()) == 0.0  # nothing was enqueued


def test_static_rejects_bad_pointers(cuda):
    import torch
    grid = small_yinyang(W)
    with Plan(grid, "fp64") as plan:
        rho = torch.ones(plan.info["n_cells"] + 2, dtype=torch.float64, device=cuda)
        phi = torch.zeros_like(rho)
        with pytest.raises(YgsError):
            ygs_solve_static(plan, rho[1:], phi)  # 8-byte offset: not 16-byte aligned
        with pytest.raises(YgsError):
            ygs_solve_static(plan, rho, rho)  # overlapping input and output
