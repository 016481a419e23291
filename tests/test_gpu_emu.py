"""The FP64-accurate split on the BF16 tensor cores (YGS_FP64_EMU) on the
cases that exercise its grids: degenerate densities, a wide dynamic range,
physical units, sign changes and the field's exponent windows, all against
the oracle at 1e-12 (the FP64 parity cases, configs 0-2 and the adjoint run in
test_gpu_fp64.py, test_gpu_config1.py, test_gpu_config2.py and
test_gpu_adjoint.py)."""
import math

import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_get_moments, ygs_solve, workloads as W
from tests._util import col_rel, rel_max, small_yinyang
from tests.test_gpu_split import _special_density, _rel_to_max

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _solve(grid, rho, **kw):
    import torch
    with Plan(grid, "fp64emu", **kw) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        B, M = ygs_get_moments(plan)
        torch.cuda.synchronize()
        return phi.cpu().numpy(), B.cpu().numpy(), M.cpu().numpy()


@pytest.mark.parametrize("kind", ["zero", "signed", "yin_equals_yang", "yang_zero"])
def test_special_densities(cuda, kind):
    """All-zero windows (zero digits, factor 2^-126), sign changes, and the
    exact cancellations sigma- = 0 or sigma+ = sigma- of the Yin-Yang sums."""
    grid = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=30, l_max=9)
    rho = _special_density(grid, kind)
    ref = oracle.solve(grid, rho)
    got, _, _ = _solve(grid, rho)
    if kind == "zero":
        assert np.all(got == 0.0)
        return
    assert _rel_to_max(got, ref) <= TOL, kind


def test_dynamic_range_across_windows(cuda):
    """Cells spanning 1e-20 .. 1e20 (so that neighbouring 256-cell windows sit
    on grids far apart): Phi to 1e-12 of the oracle, relative to its largest
    magnitude per shell (cells 1e-20 below their window's largest value carry
    no digits)."""
    grid = small_yinyang(W, n_theta=30, n_phi=88, deg=2.0, n_r=12, l_max=8)
    rng = np.random.default_rng(12)
    rho = 10.0 ** rng.uniform(-20, 20, grid.n_cells)
    ref = oracle.solve(grid, rho)
    got, _, _ = _solve(grid, rho)
    assert _rel_to_max(got, ref) <= TOL


@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_physical_units(cuda, scale):
    """G = 6.674e-8 (cgs) and densities of order 1e12 or 1e-12."""
    base = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    grid = W.yinyang_grid(13, 37, math.radians(4.0), base.edges, 9, G=6.674e-8)
    rho = W.random_density(grid, 21) * scale
    phi_ref, B_ref, M_ref = oracle.solve(grid, rho, moments=True)
    got, B, M = _solve(grid, rho)
    assert rel_max(got, phi_ref) <= TOL
    assert col_rel(B, B_ref) <= TOL
    assert col_rel(M, M_ref) <= TOL


def test_signed_density_many_windows(cuda):
    """A signed density on a 2-degree grid (Nr = 64, l_max = 24), whose
    chunks hold many 256-cell windows: every window sum is exact, so the
    error stays at the float-float flushes' level."""
    grid = small_yinyang(W, n_theta=46, n_phi=136, deg=2.0, n_r=64, l_max=24)
    rho = W.random_density(grid, 33) - 0.9
    ref = oracle.solve(grid, rho)
    got, _, _ = _solve(grid, rho)
    assert _rel_to_max(got, ref) <= TOL


def test_autotuned_split_k(cuda):
    grid = small_yinyang(W, n_theta=16, n_phi=46, deg=4.0, n_r=150, l_max=12)
    rho = W.random_density(grid, 31)
    ref = oracle.solve(grid, rho)
    got, _, _ = _solve(grid, rho, autotune=True)
    assert rel_max(got, ref) <= TOL
