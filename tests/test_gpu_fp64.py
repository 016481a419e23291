"""GPU parity of the FP64 paths against the CPU oracle (O2), through the C ABI:
the FP64 CUDA-core kernels, the FP64 tensor cores (DMMA) and the FP64-accurate
split on the BF16 tensor cores (YGS_FP64_EMU), all at 1e-12."""
import math

import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_backward, ygs_get_moments, ygs_get_weights, ygs_solve, workloads as W
from tests._util import col_rel, rel_max, rel_norm, small_yinyang

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def three_patch_grid(l_max=7):
    rng = np.random.default_rng(5)
    eul = [W.random_euler(rng) for _ in range(3)]
    nt, nf = [5, 7, 4], [11, 9, 21]
    tr = [(0.3, 2.5), (0.6, 2.2), (0.0, math.pi)]
    pr = [(-2.0, 2.4), (-1.0, 1.7), (0.0, 2 * math.pi)]
    w = rng.uniform(0.2, 1.0, sum(a * b for a, b in zip(nt, nf)))
    return W.make_grid(W.log_edges(11, 0.02), eul, nt, nf, tr, pr, l_max, G=2.5, w=w)


def hole_grid():
    return W.yinyang_grid(5, 14, math.radians(10.0), W.linear_edges(7, 0.3, 1.3), 5)


CASES = {
    "yy_small_sym": (lambda: small_yinyang(W), True),
    "yy_small_general": (lambda: small_yinyang(W), False),
    "yy_ragged": (lambda: small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9), True),
    "yy_centre_eval": (lambda: small_yinyang(W, eval=1), True),
    "polar": (lambda: W.polar_grid(7, 13, W.linear_edges(6, 0.1, 1.0), 5), True),
    "three_patch": (three_patch_grid, True),
    "hole": (hole_grid, True),
    "lmax0": (lambda: small_yinyang(W, l_max=0), True),
    "one_shell": (lambda: small_yinyang(W, n_r=1, l_max=3), True),
}


@pytest.fixture(scope="module", params=[(c, p) for c in sorted(CASES) for p in ("fp64", "fp64tc", "fp64emu")],
                ids=lambda cp: f"{cp[0]}-{cp[1]}")
def case(request, cuda):
    """Every case on the FP64 CUDA-core kernels, the FP64 tensor cores (DMMA)
    and the FP64-accurate BF16 split."""
    import torch
    name, precision = request.param
    make, sym = CASES[name]
    grid = make()
    rho = W.random_density(grid, 11)
    plan = Plan(grid, precision, symmetry=sym)
    phi_ref, B_ref, M_ref = oracle.solve(grid, rho, moments=True)
    yield f"{name}-{precision}", grid, rho, plan, phi_ref, B_ref, M_ref
    plan.close()


def test_phi_matches_oracle(case):
    import torch
    name, grid, rho, plan, phi_ref, _, _ = case
    phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    err = rel_max(phi.cpu().numpy(), phi_ref)
    assert err <= FP64_TOL, f"{name}: {err:.3e}"


def test_moments_match_oracle(case):
    import torch
    name, grid, rho, plan, _, B_ref, M_ref = case
    ygs_solve(plan, torch.from_numpy(rho).cuda())
    B, M = ygs_get_moments(plan)
    torch.cuda.synchronize()
    assert col_rel(B.cpu().numpy(), B_ref) <= 1e-12, name
    assert col_rel(M.cpu().numpy(), M_ref) <= 1e-12, name


def test_weights_match_oracle_quadrature(case):
    name, grid, rho, plan, _, _, _ = case
    if name.endswith("fp64tc") or name.endswith("fp64emu"):
        pytest.skip("the same weights as the fp64 plan")
    U_ref = oracle.build_U(grid)
    Q_ref = oracle.build_Q(grid)
    off = 0
    for p in range(grid.n_patch):
        n = grid.nang(p)
        U = ygs_get_weights(plan, "U", p)
        Q = ygs_get_weights(plan, "Q", p)
        scaleU = np.abs(U_ref).max()
        assert np.abs(U - U_ref[off:off + n]).max() <= 1e-13 * scaleU, (name, p)
        assert np.abs(Q - Q_ref[off:off + n]).max() <= 1e-13 * abs(grid.G), (name, p)
        off += n


def test_adjoint_matches_oracle_transpose(case):
    import torch
    name, grid, rho, plan, _, _, _ = case
    w = np.random.default_rng(3).standard_normal(grid.n_cells)
    got = ygs_backward(plan, torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    ref = oracle.apply_T(grid, w)
    assert rel_norm(got.cpu().numpy(), ref) <= FP64_TOL, name
    # dot-product identity <w, A rho> = <A^T w, rho>
    phi = ygs_solve(plan, torch.from_numpy(rho).cuda()).cpu().numpy()
    lhs, rhs = float(w @ phi), float(got.cpu().numpy() @ rho)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(w) @ np.abs(phi)), name


@pytest.mark.parametrize("precision", ["fp64", "fp64emu"])
def test_config0_fp64(cuda, precision):
    import torch
    grid, rho = W.config0()
    ref = oracle.solve(grid, rho)
    with Plan(grid, precision) as plan:
        assert plan.info["symmetric"] == 1
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        assert rel_max(phi.cpu().numpy(), ref) <= FP64_TOL


@pytest.mark.parametrize("precision", ["fp64", "fp64emu"])
def test_deterministic(cuda, precision):
    import torch
    grid = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    rho = torch.from_numpy(W.random_density(grid, 2)).cuda()
    with Plan(grid, precision) as plan:
        a = ygs_solve(plan, rho).clone()
        b = ygs_solve(plan, rho)
        torch.cuda.synchronize()
        assert torch.equal(a, b)
