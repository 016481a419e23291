"""Failure detection without a GPU fault: a bounded device-side wait that runs
out reports YGS_ERR_TIMEOUT through ygs_get_status and leaves the context
usable; host-injected device-allocation failures in ygs_create return
YGS_ERR_OOM and release everything allocated so far."""
import os

import numpy as np
import pytest

from paper_1903_08475_gb300 import Plan, YgsError, ygs_debug_wait_timeout, ygs_get_status, ygs_solve, workloads as W
from tests._util import small_yinyang

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout(cuda):
    import torch
    grid = small_yinyang(W)
    rho = torch.from_numpy(W.random_density(grid, 3)).cuda()
    with Plan(grid, "bf16x6") as plan:
        before = ygs_solve(plan, rho).clone()
        ygs_get_status(plan)  # clean
        ygs_debug_wait_timeout(plan, 2000)
        with pytest.raises(YgsError) as ei:
            ygs_get_status(plan)
        assert ei.value.status == 6
        ygs_get_status(plan)  # the word was read and cleared
        after = ygs_solve(plan, rho)
        torch.cuda.synchronize()
        assert torch.equal(before, after)


@pytest.mark.parametrize("precision", ["fp64", "bf16x6"])
def test_injected_allocation_failures(cuda, precision):
    import torch
    grid = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    failures = 0
    try:
        for k in (1, 2, 3, 5, 8, 13, 21, 34):
            os.environ["YGS_INJECT_ALLOC_FAILURE"] = str(k)
            try:
                Plan(grid, precision).close()
            except YgsError as e:
                assert e.status == 2, e
                failures += 1
    finally:
        os.environ.pop("YGS_INJECT_ALLOC_FAILURE", None)
    assert failures >= 4
    with Plan(grid, precision) as plan:
        assert plan.info["n_cells"] == grid.n_cells
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20  # nothing of the failed creates stays allocated


def test_create_rejects_a_wrong_rotation(cuda, monkeypatch):
    """ygs_create checks Y(R xi) = W Y(xi) (Eqs. ylm_transform, wigner-D) at
    fixed directions; a rotation table with its degree-1 block negated (the
    testing hook YGS_TEST_PERTURB_WIGNER) is caught as YGS_ERR_NUMERIC, and
    the same grid builds normally without the hook."""
    grid = small_yinyang(W)
    monkeypatch.setenv("YGS_TEST_PERTURB_WIGNER", "1")
    with pytest.raises(YgsError) as e:
        Plan(grid, "fp64")
    assert "YGS_ERR_NUMERIC" in str(e.value) and "self-check" in str(e.value)
    monkeypatch.delenv("YGS_TEST_PERTURB_WIGNER")
    with Plan(grid, "fp64") as plan:
        assert plan.info["K"] == (grid.l_max + 1) ** 2
