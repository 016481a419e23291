"""Multi-rank helpers (one process per GPU).

Two decompositions:
* replicas: solves of independent density fields shard across ranks with no
  collective on the data path (the only collectives are the timing and
  throughput reductions of a benchmark run);
* angular sharding of one field (Sect. 4.3, steps 2-3): each rank projects a
  contiguous range of the plan's split-K chunks of angular cells, the partial
  moments B (n_r x K) are summed over the ranks by one all-reduce, and every
  rank finishes the solve from the whole B.
Works with NCCL (GPU tensors) and gloo (host copies).
"""
from __future__ import annotations

import os
from typing import Tuple


def env() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous, balanced block of item indices owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(n_items, world)
    lo = rank * q + min(rank, r)
    return range(lo, lo + q + (1 if rank < r else 0))


def _reduce(x: float, op, device) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device="cpu") -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM, device)


def allreduce_moments(B, group=None):
    """Sums a moment array over the ranks in place (gloo reduces a host copy of
    a device tensor; NCCL reduces it where it is)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return B
    if B.is_cuda and dist.get_backend(group) == "gloo":
        h = B.cpu()
        dist.all_reduce(h, group=group)
        B.copy_(h)
    else:
        dist.all_reduce(B, group=group)
    return B


def angular_solve(plan, rho, out=None, group=None, stream=None):
    """Phi of one field with the angular cells sharded over the ranks of
    `group`: this rank projects its block of the plan's FP64 split-K chunks
    (ygs_project_partial), the moments are summed (allreduce_moments), and the
    solve is finished from them (ygs_finish_from_moments).  Every rank returns
    the whole Phi."""
    import torch
    import torch.distributed as dist
    from ._ygs import ygs_finish_from_moments, ygs_project_partial
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    mine = shard(plan.info["fp64_split_k"], rank, world)
    B = ygs_project_partial(plan, rho, mine.start, mine.stop, stream=stream)
    if stream is not None:
        stream.synchronize()
    else:
        torch.cuda.synchronize(rho.device)
    allreduce_moments(B, group)
    return ygs_finish_from_moments(plan, B, out, stream=stream)
