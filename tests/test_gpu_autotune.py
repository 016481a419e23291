"""Plans tuned at create (YGS_FLAG_AUTOTUNE): the projection's split-K count and
the synthesis's tile shape (full-tile width of 144, 96 or 48 shells, whole
groups of an epilogue warp's columns; one CTA per 128-cell tile or CTA pairs)
picked by timing candidates on this GPU.

Every tiling computes each output element over the same k-steps in the same
order, so the synthesis's results do not depend on the shape it runs at; a
tuned plan whose split-K count equals the untuned plan's therefore returns
the same Phi bit for bit, and any tuned plan stays within the precision's
bound of the CPU FP64 oracle (forward and adjoint).  The grids have shell
counts whose tilings differ at every candidate width (Nr = 300: 2 full tiles
and a 16-shell tail at 144, 3 and a 16-shell tail at 96, 6 and a 16-shell
tail at 48; Nr = 150: a tail narrower than a tile at each)."""
import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_backward, ygs_solve, workloads as W
from tests._util import rel_max, small_yinyang

pytestmark = pytest.mark.gpu

TOL = {"bf16x6": 1e-6, "bf16x3": 5e-4, "fp16x3": 1e-6, "tf32x3": 1e-6}
ADJ_TOL = {"bf16x6": 2e-6, "bf16x3": 5e-4, "fp16x3": 2e-6, "tf32x3": 2e-6}

CASES = {
    "nr300": lambda: small_yinyang(W, n_theta=10, n_phi=30, deg=6.0, n_r=300, l_max=6),
    "nr150_ragged": lambda: small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=150, l_max=9),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, cuda):
    grid = CASES[request.param]()
    rho = W.random_density(grid, 41)
    return request.param, grid, rho, oracle.solve(grid, rho)


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "bf16x6", "tf32x3"])
def test_tuned_tile_shape_matches_oracle(case, precision):
    import torch
    name, grid, rho, phi_ref = case
    r = torch.from_numpy(rho).cuda()
    with Plan(grid, precision, autotune=True) as pt, Plan(grid, precision) as p0:
        w = pt.info["synth_tile_shells"]
        assert w in (48, 96, 144), w
        assert p0.info["synth_tile_shells"] == 144 and p0.info["cta_pairs"] == 0
        a = ygs_solve(pt, r)
        torch.cuda.synchronize()
        err = rel_max(a.cpu().numpy(), phi_ref)
        assert err <= TOL[precision], f"{name} {precision} (w {w}, pairs {pt.info['cta_pairs']}): {err:.3e}"
        if pt.info["split_k"] == p0.info["split_k"]:
            b = ygs_solve(p0, r)
            torch.cuda.synchronize()
            assert torch.equal(a, b), f"{name} {precision}: tuned tile shape (w {w}) changed Phi " \
                                      f"({float((a - b).abs().max()):.3e})"


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x6"])
def test_tuned_adjoint_matches_oracle_transpose(case, precision):
    import torch
    name, grid, _, _ = case
    g = W.random_density(grid, 7)
    ref = oracle.apply_T(grid, g)
    with Plan(grid, precision, autotune=True) as pt:
        got = ygs_backward(pt, torch.from_numpy(g).cuda())
        torch.cuda.synchronize()
        err = rel_max(got.cpu().numpy(), ref)
        assert err <= ADJ_TOL[precision], f"{name} {precision}: {err:.3e}"


def test_fp64_accurate_plan_keeps_its_synthesis_shape(cuda):
    grid = small_yinyang(W, n_r=40)
    with Plan(grid, "fp64emu", autotune=True) as p:
        assert p.info["synth_tile_shells"] == 128 and p.info["cta_pairs"] == 0
    with Plan(grid, "fp64", autotune=True) as p:
        assert p.info["synth_tile_shells"] == 0
