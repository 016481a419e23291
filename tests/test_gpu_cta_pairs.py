"""The split-precision synthesis on CTA pairs (cta_group::2: one 256-cell tile
per cluster of two CTAs, the even CTA issuing every MMA for both, each CTA
staging its own 128 cells of Q and half of the tile's shells of M) against
the default single-CTA synthesis and the CPU FP64 oracle (YGS_FLAG_CTA_PAIRS).

The two launch shapes accumulate every output element over the same k-steps
in the same order, so Phi (and the adjoint's grad_rho) agree bit for bit.
Cases cover a ragged last pair tile (cells of the odd CTA past the patch), a
tail shell tile (half of it per CTA), one shell, and patches without the
Yin-Yang symmetry (one column block)."""
import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_backward, ygs_solve, workloads as W
from tests._util import rel_max, small_yinyang

pytestmark = pytest.mark.gpu

TOL = {"bf16x6": 1e-6, "bf16x3": 5e-4, "fp16x3": 1e-6, "tf32x3": 1e-6}

CASES = {
    # 108 cells per patch: one pair tile, the odd CTA's cells all past the patch
    "yy_small": lambda: small_yinyang(W),
    # 481 cells per patch: the last pair tile ragged inside the odd CTA
    "yy_ragged": lambda: small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9),
    # 150 shells: one full 144-shell tile and a 16-shell tail (8 shells per CTA)
    "shell_tail": lambda: small_yinyang(W, n_theta=10, n_phi=30, deg=6.0, n_r=150, l_max=6),
    "one_shell": lambda: small_yinyang(W, n_r=1, l_max=3),
    "polar": lambda: W.polar_grid(7, 13, W.linear_edges(6, 0.1, 1.0), 5),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, cuda):
    grid = CASES[request.param]()
    rho = W.random_density(grid, 23)
    return request.param, grid, rho, oracle.solve(grid, rho)


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "bf16x6", "tf32x3"])
def test_pairs_equal_single_cta_and_match_oracle(case, precision):
    import torch
    name, grid, rho, phi_ref = case
    r = torch.from_numpy(rho).cuda()
    with Plan(grid, precision, cta_pairs=True) as pp, Plan(grid, precision) as ps:
        assert pp.info["cta_pairs"] == 1 and ps.info["cta_pairs"] == 0
        a = ygs_solve(pp, r)
        b = ygs_solve(ps, r)
        torch.cuda.synchronize()
        assert torch.equal(a, b), f"{name} {precision}: pair and single-CTA synthesis differ " \
                                  f"({float((a - b).abs().max()):.3e})"
        err = rel_max(a.cpu().numpy(), phi_ref)
        assert err <= TOL[precision], f"{name} {precision}: {err:.3e}"


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x6"])
def test_adjoint_pairs_equal_single_cta(case, precision):
    import torch
    name, grid, rho, _ = case
    g = torch.from_numpy(W.random_density(grid, 5)).cuda()
    with Plan(grid, precision, cta_pairs=True) as pp, Plan(grid, precision) as ps:
        a = ygs_backward(pp, g)
        b = ygs_backward(ps, g)
        torch.cuda.synchronize()
        assert torch.equal(a, b), f"{name} {precision}: {float((a - b).abs().max()):.3e}"
        ref = oracle.apply_T(grid, g.cpu().numpy())
        assert rel_max(a.cpu().numpy(), ref) <= 2e-6


def test_fp64_accurate_and_fp64_plans_run_single_cta(cuda):
    grid = small_yinyang(W)
    for precision in ("fp64emu", "fp64"):
        with Plan(grid, precision, cta_pairs=True) as p:
            assert p.info["cta_pairs"] == 0
