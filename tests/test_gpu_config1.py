"""Full-size Yin-Yang 1 degree grid (Nr = 400, l_max = 32): GPU Phi on sampled
cells against the oracle evaluated cell by cell."""
import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_get_moments, ygs_solve, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1():
    grid, rho = W.config1()
    U = oracle.build_U(grid)
    B = oracle.project(grid, rho, U)
    M = oracle.radial(grid, B)
    Q = oracle.build_Q(grid)
    return grid, rho, B, M, Q


def sample_phi(grid, M, Q, idx):
    out = np.empty(len(idx))
    na = grid.nang(0)
    for n, e in enumerate(idx):
        g, rem = divmod(int(e), grid.n_r * na)
        i, a = divmod(rem, na)
        out[n] = Q[g * na + a] @ M[i]
    return out


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp64tc", 1e-12), ("fp64emu", 1e-12), ("bf16x6", 1e-6), ("fp16x3", 1e-6), ("tf32x3", 1e-6), ("fp32", 1e-4)])
def test_config1_sampled(cfg1, cuda, precision, tol):
    import torch
    grid, rho, B_ref, M_ref, Q = cfg1
    with Plan(grid, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        B, M = ygs_get_moments(plan)
        torch.cuda.synchronize()
        phi = phi.cpu().numpy()
    idx = np.random.default_rng(0).choice(grid.n_cells, 4000, replace=False)
    ref = sample_phi(grid, M_ref, Q, idx)
    err = np.max(np.abs(phi[idx] - ref) / np.abs(ref))
    assert err <= tol, err
    Bc = B.cpu().numpy()
    assert np.abs(Bc[:, 0] / B_ref[:, 0] - 1).max() <= tol
