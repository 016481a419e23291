"""Batched solves and CUDA-graph capture through the C ABI."""
import math

import numpy as np
import pytest

from paper_1903_08475_gb300 import Batch, Plan, YgsError, ygs_solve, ygs_solve_batched, workloads as W
from tests._util import small_yinyang
from tests.test_gpu_fp64 import three_patch_grid

pytestmark = pytest.mark.gpu


def _fields(cuda):
    import torch
    grids = [small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9),
             small_yinyang(W, n_theta=8, n_phi=20, n_r=150, l_max=7),
             three_patch_grid(),
             W.polar_grid(7, 13, W.linear_edges(6, 0.1, 1.0), 5)]
    precs = ["bf16x6", "fp64", "fp16x3", "bf16x3"]
    plans = [Plan(g, p) for g, p in zip(grids, precs)]
    rhos = [torch.from_numpy(W.random_density(g, 20 + i)).cuda() for i, g in enumerate(grids)]
    return plans, rhos


def test_batched_equals_per_field(cuda):
    import torch
    plans, rhos = _fields(cuda)
    ref = [ygs_solve(p, r).clone() for p, r in zip(plans, rhos)]
    # the first plan twice: same workspaces, kept in order on one worker stream
    bp = plans + [plans[0]]
    br = rhos + [rhos[0] * 2.0]
    outs = [torch.empty_like(r) for r in br]
    ygs_solve_batched(bp, br, outs)
    torch.cuda.synchronize()
    for a, b in zip(ref, outs[:-1]):
        assert torch.equal(a, b)
    assert torch.allclose(outs[-1], 2.0 * ref[0], rtol=1e-6, atol=0)
    for p in plans:
        p.close()


def test_graph_capture_single_and_batched(cuda):
    import torch
    plans, rhos = _fields(cuda)
    outs = [torch.empty_like(r) for r in rhos]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ygs_solve_batched(plans, rhos, outs, stream=s)  # warm-up outside the capture
        ygs_solve(plans[0], rhos[0], outs[0], stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [o.clone() for o in outs]
    g1 = torch.cuda.CUDAGraph()
    single = torch.empty_like(rhos[0])
    with torch.cuda.graph(g1):
        ygs_solve(plans[0], rhos[0], single)
    g2 = torch.cuda.CUDAGraph()
    gouts = [torch.empty_like(r) for r in rhos]
    with torch.cuda.graph(g2):
        ygs_solve_batched(plans, rhos, gouts)
    for _ in range(2):
        g1.replay()
        g2.replay()
    torch.cuda.synchronize()
    assert torch.equal(single, eager[0])
    for a, b in zip(gouts, eager):
        assert torch.equal(a, b)
    for p in plans:
        p.close()


def _uneven_fields(cuda):
    """Split-precision and FP64 plans of different sizes, patch sets and l_max."""
    import torch
    grids = [small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9),
             small_yinyang(W, n_theta=8, n_phi=20, n_r=150, l_max=7),
             three_patch_grid(),
             W.polar_grid(7, 13, W.linear_edges(6, 0.1, 1.0), 5),
             small_yinyang(W, n_theta=10, n_phi=28, n_r=300, l_max=12),
             small_yinyang(W, n_theta=6, n_phi=18, n_r=9, l_max=0),
             small_yinyang(W, n_theta=9, n_phi=25, n_r=40, l_max=8)]
    precs = ["fp16x3", "bf16x6", "tf32x3", "fp64", "bf16x3", "fp16x3", "fp64emu"]
    plans = [Plan(g, p) for g, p in zip(grids, precs)]
    rhos = [torch.from_numpy(W.random_density(g, 40 + i)).cuda() for i, g in enumerate(grids)]
    return plans, rhos


def test_grouped_batch_equals_per_field(cuda):
    """One persistent launch per operand kind for the contractions of every
    field gives bit-identical results to the per-field solves."""
    import torch
    plans, rhos = _uneven_fields(cuda)
    ref = [ygs_solve(p, r).clone() for p, r in zip(plans, rhos)]
    with Batch(plans) as b:
        # 7 fields in five operand kinds (FP16 two-slice, BF16 two-slice, BF16
        # three-slice, TF32 two-slice, EMU six-slice): per kind one grouped
        # launch each for the field slices, the projection, the scans (+ the M
        # slicing for FP16 and EMU) and the synthesis; 3 for the FP64 field
        assert b.launches == 5 + 4 + 4 + 4 + 5 + 3
        for _ in range(2):
            outs = b.solve(rhos)
            torch.cuda.synchronize()
            for a, o in zip(ref, outs):
                assert torch.equal(a, o)
    for p in plans:
        p.close()


def test_grouped_batch_in_a_cuda_graph(cuda):
    import torch
    plans, rhos = _uneven_fields(cuda)
    ref = [ygs_solve(p, r).clone() for p, r in zip(plans, rhos)]
    with Batch(plans) as b:
        outs = [torch.empty_like(r) for r in rhos]
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            b.solve(rhos, outs, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        gin = [r.clone() for r in rhos]
        gout = [torch.empty_like(r) for r in rhos]
        with torch.cuda.graph(g):
            b.solve(gin, gout)
        for k, r in enumerate(rhos):  # new inputs into the captured buffers
            gin[k].copy_(2.0 * r)
        g.replay()
        torch.cuda.synchronize()
        for a, o in zip(ref, gout):
            assert torch.allclose(o, 2.0 * a, rtol=1e-6, atol=0)
    for p in plans:
        p.close()


def test_batch_rejects_repeated_plan(cuda):
    plans, _ = _uneven_fields(cuda)
    with pytest.raises(YgsError):
        Batch([plans[0], plans[1], plans[0]])
    for p in plans:
        p.close()


@pytest.mark.parametrize("precision", ["fp16x3", "fp64"])
def test_solve_host_many_equals_device_solves(cuda, precision):
    """The pipelined host-buffer entry point (uploads, solves and read-backs
    of consecutive fields overlapped through two staging pairs) gives, field
    by field, the same bits as ygs_solve on device buffers; n = 0 and n = 1
    included."""
    import torch
    from paper_1903_08475_gb300 import ygs_solve_host_many
    grid = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    fields = [W.random_density(grid, 60 + k) * (1.0 + k) for k in range(5)]
    with Plan(grid, precision) as plan:
        ref = [ygs_solve(plan, torch.from_numpy(f).cuda()).cpu() for f in fields]
        torch.cuda.synchronize()
        for n in (0, 1, 5):
            h_rho = [torch.from_numpy(f).pin_memory() for f in fields[:n]]
            h_phi = [torch.empty_like(r).pin_memory() for r in h_rho]
            ygs_solve_host_many(plan, h_rho, h_phi)
            for k in range(n):
                assert torch.equal(h_phi[k], ref[k]), (n, k)
        with pytest.raises(ValueError):
            ygs_solve_host_many(plan, [torch.zeros(1)], [])
