"""The hand-written adjoint (ygs_backward, the autograd backward of
paper_1903_08475_gb300.potential): central finite differences, autograd, and
the oracle's transposed operator at the full adjoint workload (Yin-Yang 1
degree, Nr = 256, l_max = 32)."""
import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, potential, ygs_backward, ygs_solve, workloads as W
from tests._util import rel_norm, small_yinyang

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp64emu", 1e-10), ("bf16x6", 1e-6), ("fp16x3", 1e-6),
                                           ("tf32x3", 1e-6)])
def test_central_differences_on_64_cells(cuda, precision, tol):
    """J(rho) = sum w Phi(rho) is linear: (J(rho + h e_k) - J(rho - h e_k)) / 2h
    equals (A^T w)_k.  Phi is differenced elementwise before the dot product,
    with h large enough that the impulse dominates the field."""
    import torch
    grid = small_yinyang(W, n_theta=10, n_phi=28, n_r=40, l_max=10)
    rho = W.random_density(grid, 5)
    w = torch.from_numpy(np.random.default_rng(6).standard_normal(grid.n_cells)).cuda()
    cells = np.random.default_rng(7).choice(grid.n_cells, 64, replace=False)
    with Plan(grid, precision) as plan, Plan(grid, "fp64") as p64:
        g = ygs_backward(p64, w).cpu().numpy()
        # the plan's own adjoint (tensor cores for split precisions) against the FP64 one
        gs = ygs_backward(plan, w).cpu().numpy()
        assert np.max(np.abs(gs - g)) <= tol * np.max(np.abs(g)), precision
        base = torch.from_numpy(rho).cuda()
        h = 1e8
        for k in cells:
            up, dn = base.clone(), base.clone()
            up[k] += h
            dn[k] -= h
            d = (ygs_solve(plan, up) - ygs_solve(plan, dn)) / (2 * h)
            fd = float((w * d).sum())
            assert abs(fd - g[k]) <= tol * max(abs(g[k]), float((w.abs() * d.abs()).sum())), (k, fd, g[k])


def test_autograd_matches_backward(cuda):
    import torch
    grid = small_yinyang(W, n_theta=8, n_phi=24, n_r=20, l_max=8)
    rho = torch.from_numpy(W.random_density(grid, 8)).cuda().requires_grad_(True)
    w = torch.from_numpy(np.random.default_rng(9).standard_normal(grid.n_cells)).cuda()
    with Plan(grid, "bf16x6") as plan:
        J = (w * potential(rho, plan)).sum()
        J.backward()
        ref = ygs_backward(plan, w)
        torch.cuda.synchronize()
        assert torch.equal(rho.grad, ref)


@pytest.fixture(scope="module")
def config4_transpose():
    grid, rho, w = W.config4()
    U = oracle.build_U(grid)
    Q = oracle.build_Q(grid)
    return grid, rho, w, oracle.apply_T(grid, w, U=U, Q=Q)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp64emu", 1e-12), ("bf16x6", 1e-6), ("fp16x3", 1e-6),
                                           ("tf32x3", 1e-6)])
def test_adjoint_full_size_vs_oracle_transpose(cuda, config4_transpose, precision, tol):
    """Yin-Yang 1 degree, Nr = 256, l_max = 32, w ~ N(0, 1): the plan's adjoint
    (FP64 kernels, or the tensor cores for split precisions) against the
    oracle's transposed loops.  TF32x3 has the same 22-bit operands as FP16x3,
    but the kind::tf32 MMA takes K = 8 per instruction, so its accumulator is
    rounded twice as often per k: flushed every 64 k like the others its
    adjoint reached 1.4e-6 of the largest |A^T w|, so the TF32 adjoint flushes
    every k-block (32 k)."""
    import torch
    grid, rho, w, ref = config4_transpose
    with Plan(grid, precision) as plan:
        got = ygs_backward(plan, torch.from_numpy(w).cuda()).cpu().numpy()
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda()).cpu().numpy()
    assert rel_norm(got, ref) <= tol
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    # dot-product identity <w, A rho> = <A^T w, rho>
    assert abs(w @ phi - got @ rho) <= tol * (np.abs(w) @ np.abs(phi))
