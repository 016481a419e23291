"""Angular sharding of one field (Sect. 4.3, steps 2-3) through the C ABI:
partial projections over ranges of the FP64 split-K chunks, the moments
summed, the solve finished from them; and two gloo ranks on one device doing
the same through paper_1903_08475_gb300.dist (their kernels never wait on each
other: the exchange is one host all-reduce between the two calls)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import (Plan, YgsError, ygs_finish_from_moments, ygs_get_moments, ygs_project_partial,
                                    ygs_solve, workloads as W)
from paper_1903_08475_gb300 import dist as D
from tests._util import rel_max, small_yinyang
from tests.test_gpu_fp64 import three_patch_grid

pytestmark = pytest.mark.gpu


def _grid():
    return small_yinyang(W, n_theta=16, n_phi=46, deg=4.0, n_r=40, l_max=10)


@pytest.mark.parametrize("make,precision", [(_grid, "fp64"), (_grid, "fp64tc"), (three_patch_grid, "fp64"),
                                            (_grid, "fp16x3")])
def test_partial_projections_sum_to_the_solve(cuda, make, precision):
    import torch
    grid = make()
    rho = torch.from_numpy(W.random_density(grid, 7)).cuda()
    ref = oracle.solve(grid, rho.cpu().numpy())
    with Plan(grid, precision) as plan:
        S = plan.info["fp64_split_k"]
        assert S >= 3, S
        cuts = [0, S // 3, (2 * S) // 3, S]
        B = sum(ygs_project_partial(plan, rho, a, b) for a, b in zip(cuts, cuts[1:]))
        phi = ygs_finish_from_moments(plan, B)
        torch.cuda.synchronize()
        assert rel_max(phi.cpu().numpy(), ref) <= 1e-12
        if precision != "fp16x3":
            phi1 = ygs_solve(plan, rho)
            B1, _ = ygs_get_moments(plan)
            torch.cuda.synchronize()
            assert rel_max(phi.cpu().numpy(), phi1.cpu().numpy()) <= 1e-13
            assert float((B - B1).abs().max()) <= 1e-13 * float(B1.abs().max())


def test_partial_projection_edges(cuda):
    import torch
    grid = _grid()
    rho = torch.from_numpy(W.random_density(grid, 8)).cuda()
    with Plan(grid, "fp64") as plan:
        S = plan.info["fp64_split_k"]
        Z = ygs_project_partial(plan, rho, 1, 1)
        torch.cuda.synchronize()
        assert float(Z.abs().max()) == 0.0
        for a, b in [(-1, 1), (2, 1), (0, S + 1)]:
            with pytest.raises(YgsError):
                ygs_project_partial(plan, rho, a, b)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = _grid()
        rho = torch.from_numpy(W.random_density(grid, 9)).cuda()
        with Plan(grid, "fp64") as plan:
            phi = D.angular_solve(plan, rho)
            torch.cuda.synchronize()
            q.put((rank, plan.info["fp64_split_k"], phi.cpu().numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_angular_solve(cuda):
    """Each rank projects half the chunks; gloo sums the partial B; both
    ranks' Phi equal the single-rank solve to 1e-12."""
    import torch
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    grid = _grid()
    rho = W.random_density(grid, 9)
    with Plan(grid, "fp64") as plan:
        ref = ygs_solve(plan, torch.from_numpy(rho).cuda()).cpu().numpy()
    assert res[0][1] >= 2
    for _, _, phi in res:
        assert rel_max(phi, ref) <= 1e-12
    assert rel_max(res[0][2], oracle.solve(grid, rho)) <= 1e-12
