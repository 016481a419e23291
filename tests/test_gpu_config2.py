"""The 0.5 degree Yin-Yang grid at l_max = 64 (184 x 544 cells per patch):
GPU against the oracle on the full angular grid with a reduced set of shells
(the oracle projection over all 800 shells takes minutes on the host), with
the error reported per l band."""
import math

import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_get_moments, ygs_solve, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg2_small():
    n_theta, n_phi, d = 184, 544, math.radians(1.0)
    edges = W.log_edges(800, 1e-3, 1.0)[::40]  # 20 shells spanning the same radii
    grid = W.yinyang_grid(n_theta, n_phi, d, edges, 64)
    rho = W.lognormal_density(grid, np.random.default_rng(W.SEED_BASE + 2), n_fft=128)
    phi, B, M = oracle.solve(grid, rho, moments=True)
    return grid, rho, phi, B, M


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp64tc", 1e-12), ("fp64emu", 1e-12), ("bf16x6", 1e-6), ("fp16x3", 1e-6), ("fp32", 1e-4)])
def test_config2_lmax64(cfg2_small, cuda, precision, tol):
    import torch
    grid, rho, phi_ref, B_ref, M_ref = cfg2_small
    with Plan(grid, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        B, M = ygs_get_moments(plan)
        torch.cuda.synchronize()
        phi = phi.cpu().numpy()
        B = B.cpu().numpy()
    err = float(np.max(np.abs(phi - phi_ref) / np.abs(phi_ref)))
    assert err <= tol, err
    # per-l band error of the moments B (relative 2-norm of the columns of each degree)
    bands = []
    for l in range(grid.l_max + 1):
        cols = slice(l * l, (l + 1) * (l + 1))
        bands.append(np.linalg.norm(B[:, cols] - B_ref[:, cols]) / max(np.linalg.norm(B_ref[:, cols]), 1e-300))
    print(f"{precision}: max rel Phi err {err:.2e}; B error per l band: "
          + " ".join(f"{b:.1e}" for b in bands[::8]))
    assert bands[0] <= tol
