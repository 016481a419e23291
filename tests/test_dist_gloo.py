"""The multi-rank host logic on CPU: two gloo ranks shard a batch of fields
and reduce timings the way a multi-GPU benchmark run does."""
import os
import socket

import pytest

from paper_1903_08475_gb300 import dist as D


def test_shard_partitions_items():
    for n in (0, 1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in D.shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(D.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, rk, _ = D.env()
        mine = list(D.shard(64, rk, ws))
        # each rank "times" its own fields; the job time is the slowest rank's
        t = 1.0 + 0.5 * rk
        q.put((rk, mine, D.max_over_ranks(t), D.sum_over_ranks(len(mine))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, f0, m0, s0), (r1, f1, m1, s1) = res
    assert (r0, r1) == (0, 1)
    assert sorted(f0 + f1) == list(range(64)) and not set(f0) & set(f1)
    assert m0 == m1 == 1.5
    assert s0 == s1 == 64


def _angular_worker(rank, world, port, q):
    """One rank of an angularly sharded solve on CPU: the oracle's moments of
    this rank's block of angular cells, summed over the ranks by gloo."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1903_08475_gb300 import workloads as W
    from tests._util import small_yinyang
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid = small_yinyang(W, n_theta=7, n_phi=19, n_r=6, l_max=4)
        rho = W.random_density(grid, 3)
        mask = np.zeros(grid.n_cells)
        off = 0
        for g in range(grid.n_patch):
            na = grid.nang(g)
            cells = D.shard(na, rank, world)
            for i in range(grid.n_r):
                mask[off + i * na + cells.start: off + i * na + cells.stop] = 1.0
            off += grid.n_r * na
        U = oracle.build_U(grid)
        B = torch.from_numpy(oracle.project(grid, rho * mask, U))
        D.allreduce_moments(B)
        q.put((rank, B.numpy()))
    finally:
        dist.destroy_process_group()


def test_angular_shard_moments_two_gloo_ranks():
    """Sect. 4.3 steps 2-3 on CPU: two ranks' partial moments (disjoint blocks
    of every patch's angular cells) summed by one all-reduce equal the whole
    field's moments, and Phi finished from them equals the oracle's solve."""
    import numpy as np
    import torch.multiprocessing as mp
    import oracle
    from paper_1903_08475_gb300 import workloads as W
    from tests._util import small_yinyang
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_angular_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    grid = small_yinyang(W, n_theta=7, n_phi=19, n_r=6, l_max=4)
    rho = W.random_density(grid, 3)
    phi_ref, B_ref, M_ref = oracle.solve(grid, rho, moments=True)
    for _, B in res:
        assert np.abs(B - B_ref).max() <= 1e-13 * np.abs(B_ref).max()
    M = oracle.radial(grid, res[0][1])
    phi = oracle.synthesize(grid, M, oracle.build_Q(grid))
    assert np.max(np.abs(phi - phi_ref) / np.abs(phi_ref)) <= 1e-12
