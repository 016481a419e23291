"""The paper's own test (Sect. 5.1): a homogeneous tri-axial ellipsoid
(a, b, c) = (1, 1.5, 2), its shortest axis tilted by pi/8 from the Yin xi-axis
in the xi-eta plane, on the 1 degree Yin-Yang grid with 800 equidistant
shells in [0, 2]; maximum relative error of Phi against the closed form (the
oracle's Carlson evaluation of Eq. phiana) as a function of l_max.  The
paper's curve (Fig. 5) is not reproduced in its text, so this checks the
behaviour it describes: the error falls quickly with l_max and levels off
where the spatial discretisation dominates (the density is 1 at cells whose
centre lies inside the surface)."""
import math

import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_solve, workloads as W

pytestmark = pytest.mark.gpu

AXES = (1.0, 1.5, 2.0)
TILT = math.pi / 8


def _rz(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


@pytest.fixture(scope="module")
def setup():
    nt, nf, d = W.yinyang_resolution(1.0)
    grid = W.yinyang_grid(nt, nf, d, W.linear_edges(800, 0.0, 2.0), 8)
    # body coordinates (X, Y, Z) = Rz(pi/8) xi_Yin, so x = R_Yin Rz(pi/8)^T (X, Y, Z)
    body = W.rotation_matrix(*grid.euler[0]) @ _rz(TILT).T
    rho = W.ellipsoid_density(grid, AXES, body_rot=body, nsub=1)
    # sample of evaluation points: the Yin equatorial cut at every shell, plus random cells
    rng = np.random.default_rng(20190320)
    na = grid.nang(0)
    j_eq = grid.n_theta[0] // 2
    eq = [(0, i, j_eq * grid.n_phi[0] + k) for i in range(0, grid.n_r, 4) for k in range(0, grid.n_phi[0], 2)]
    rnd = [(int(p), int(i), int(a)) for p, i, a in zip(rng.integers(0, 2, 6000), rng.integers(0, grid.n_r, 6000),
                                                        rng.integers(0, na, 6000))]
    pts = eq + rnd
    idx = np.array([grid.patch_offset(p) + i * na + a for p, i, a in pts])
    # upper vertices (r_i^+, theta_j^+, phi_k^+) in body coordinates
    xs = []
    for p, i, a in pts:
        j, k = divmod(a, int(grid.n_phi[p]))
        th = grid.theta_range[p][0] + (j + 1) * (grid.theta_range[p][1] - grid.theta_range[p][0]) / grid.n_theta[p]
        ph = grid.phi_range[p][0] + (k + 1) * (grid.phi_range[p][1] - grid.phi_range[p][0]) / grid.n_phi[p]
        loc = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        xs.append(grid.edges[i + 1] * (W.rotation_matrix(*grid.euler[p]) @ loc))
    xb = np.array(xs) @ body  # rows: body coordinates
    ana = oracle.ellipsoid_phi(*AXES, xb[:, 0], xb[:, 1], xb[:, 2])
    return grid, rho, idx, ana


def _max_err(grid, rho, idx, ana, l_max, precision="fp64"):
    import torch
    with Plan(grid.with_lmax(l_max), precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        return float(np.max(np.abs(phi.cpu().numpy()[idx] - ana) / np.abs(ana))), phi.cpu().numpy()


def test_error_versus_lmax(cuda, setup):
    grid, rho, idx, ana = setup
    errs = {}
    for l_max in (4, 8, 16, 32, 48, 64, 80):
        errs[l_max], _ = _max_err(grid, rho, idx, ana, l_max)
    print("max relative error vs l_max: " + ", ".join(f"{l}: {e:.2e}" for l, e in errs.items()))
    # falls quickly at low order ...
    assert errs[16] < 0.5 * errs[4] and errs[32] < errs[16]
    # ... and levels off where the surface's discretisation dominates
    assert errs[80] <= errs[32]
    assert abs(errs[80] - errs[64]) <= 0.25 * errs[64]
    assert errs[80] < 2e-2


@pytest.mark.parametrize("precision", ["bf16x6", "fp16x3"])
def test_split_precision_at_lmax80(cuda, setup, precision):
    """At the paper's l_max = 80 (6561 columns) the split tensor-core path stays
    within 1e-6 of the FP64 path on the whole grid."""
    grid, rho, idx, ana = setup
    _, ref = _max_err(grid, rho, idx, ana, 80)
    _, got = _max_err(grid, rho, idx, ana, 80, precision)
    assert float(np.max(np.abs(got - ref) / np.abs(ref))) <= 1e-6
