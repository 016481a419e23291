"""GPU parity of the split-precision tensor-core path (BF16 or FP16 slices on
tcgen05) against the CPU FP64 oracle, through the C ABI.

BF16x6 (three slices, six products) and FP16x3 (two power-of-two-scaled FP16
slices, three products) are held to 1e-6 relative error in Phi; BF16x3 (two
slices, three products) to 5e-4.  The FP32 accumulation of the tensor cores
is flushed into float-float sums every 64 or 128 k-elements (128 where the
summed terms change sign and the monopole is summed exactly elsewhere), which
keeps its bias far below these bounds."""
import math

import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_get_moments, ygs_solve, workloads as W
from tests._util import rel_max, small_yinyang
from tests.test_gpu_fp64 import three_patch_grid, hole_grid

pytestmark = pytest.mark.gpu

TOL = {"bf16x6": 1e-6, "bf16x3": 5e-4, "fp16x3": 1e-6, "tf32x3": 1e-6}

CASES = {
    "yy_small": lambda: small_yinyang(W),
    "yy_ragged": lambda: small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9),
    "yy_centre_eval": lambda: small_yinyang(W, eval=1),
    "polar": lambda: W.polar_grid(7, 13, W.linear_edges(6, 0.1, 1.0), 5),
    "three_patch": three_patch_grid,
    "hole": hole_grid,
    "lmax0": lambda: small_yinyang(W, l_max=0),
    "one_shell": lambda: small_yinyang(W, n_r=1, l_max=3),
    "many_shells": lambda: small_yinyang(W, n_theta=8, n_phi=20, n_r=300, l_max=7),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, cuda):
    grid = CASES[request.param]()
    rho = W.random_density(grid, 11)
    phi_ref, B_ref, M_ref = oracle.solve(grid, rho, moments=True)
    return request.param, grid, rho, phi_ref, B_ref, M_ref


@pytest.mark.parametrize("precision", ["bf16x6", "bf16x3", "fp16x3", "tf32x3"])
def test_phi_matches_oracle(case, precision):
    import torch
    name, grid, rho, phi_ref, B_ref, M_ref = case
    with Plan(grid, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        B, M = ygs_get_moments(plan)
        torch.cuda.synchronize()
        err = rel_max(phi.cpu().numpy(), phi_ref)
        assert err <= TOL[precision], f"{name} {precision}: {err:.3e}"
        # monopole moments (all-positive sums) to the same bound
        assert rel_max(B.cpu().numpy()[:, 0], B_ref[:, 0]) <= TOL[precision]
        assert rel_max(M.cpu().numpy()[:, 0], M_ref[:, 0]) <= TOL[precision]


@pytest.mark.parametrize("precision", ["bf16x6", "fp16x3", "tf32x3"])
def test_config0(cuda, precision):
    import torch
    grid, rho = W.config0()
    ref = oracle.solve(grid, rho)
    with Plan(grid, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        assert rel_max(phi.cpu().numpy(), ref) <= TOL[precision]


def test_split_deterministic(cuda):
    import torch
    grid = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    rho = torch.from_numpy(W.random_density(grid, 2)).cuda()
    with Plan(grid, "bf16x6") as plan:
        a = ygs_solve(plan, rho).clone()
        b = ygs_solve(plan, rho)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["bf16x6", "fp16x3", "tf32x3"])
def test_large_dynamic_range(cuda, precision):
    """Density spanning 1e-30 .. 1e30 (BF16's exponent range covers it; FP16
    rows are scaled by powers of two, and cells far below a row's largest
    value contribute below the tolerance)."""
    import torch
    grid = small_yinyang(W, n_theta=8, n_phi=24, n_r=20, l_max=6)
    rng = np.random.default_rng(4)
    rho = 10.0 ** rng.uniform(-30, 30, grid.n_cells)
    ref = oracle.solve(grid, rho)
    with Plan(grid, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        assert rel_max(phi.cpu().numpy(), ref) <= TOL[precision]


@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_fp16_scaling_physical_units(cuda, scale):
    """FP16 slices outside FP16's own range: G = 6.674e-8 (cgs) and densities
    of order 1e12 or 1e-12 are brought into range by the per-row powers of two."""
    import torch
    base = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    grid = W.yinyang_grid(13, 37, math.radians(4.0), base.edges, 9, G=6.674e-8)
    rho = W.random_density(grid, 21) * scale
    ref = oracle.solve(grid, rho)
    with Plan(grid, "fp16x3") as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        assert rel_max(phi.cpu().numpy(), ref) <= TOL["fp16x3"]


@pytest.mark.parametrize("precision", ["bf16x6", "fp16x3", "tf32x3"])
def test_autotuned_split_k(cuda, precision):
    """A plan whose split-K count was picked by timing candidates at create
    (YGS_FLAG_AUTOTUNE) stays within the precision's bound of the oracle."""
    import torch
    grid = small_yinyang(W, n_theta=16, n_phi=46, deg=4.0, n_r=150, l_max=12)
    rho = W.random_density(grid, 31)
    ref = oracle.solve(grid, rho)
    with Plan(grid, precision) as p0, Plan(grid, precision, autotune=True) as p1:
        assert p1.info["split_k"] >= 1
        for p in (p0, p1):
            phi = ygs_solve(p, torch.from_numpy(rho).cuda())
            torch.cuda.synchronize()
            assert rel_max(phi.cpu().numpy(), ref) <= TOL[precision]


@pytest.mark.parametrize("name", ["yy_ragged", "three_patch", "many_shells"])
def test_fp32_cuda_core_variant(cuda, name):
    """YGS_FP32: FP32 contractions on the CUDA cores with FP64 scans; its error
    against the oracle is that of FP32 accumulation (stated, held to 1e-4)."""
    import torch
    grid = CASES[name]()
    rho = W.random_density(grid, 17)
    ref = oracle.solve(grid, rho)
    with Plan(grid, "fp32") as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        err = rel_max(phi.cpu().numpy(), ref)
    print(f"fp32 {name}: {err:.2e}")
    assert err <= 1e-4


def _rel_to_max(got, ref):
    """Largest error relative to the largest |ref| (for fields that cross zero)."""
    return float(np.max(np.abs(np.asarray(got) - ref)) / np.max(np.abs(ref)))


def _special_density(grid, kind):
    rng = np.random.default_rng(8)
    n0 = grid.n_r * grid.nang(0)
    if kind == "zero":
        return np.zeros(grid.n_cells)
    if kind == "signed":  # sums that change sign: the monopole's partials do not dominate
        return rng.standard_normal(grid.n_cells)
    yin = rng.uniform(0.5, 1.5, n0)
    if kind == "yin_equals_yang":  # sigma- = 0 in every chunk
        return np.concatenate([yin, yin])
    if kind == "yang_zero":  # sigma+ = sigma- = rho_Yin
        return np.concatenate([yin, np.zeros(grid.n_cells - n0)])
    raise ValueError(kind)


@pytest.mark.parametrize("precision", ["bf16x6", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("kind", ["zero", "signed", "yin_equals_yang", "yang_zero"])
def test_special_densities(cuda, precision, kind):
    """Densities that reach the degenerate branches of the split path: all zero
    (every scale exponent from a zero maximum, Phi exactly zero), signed
    (monopole partials of both signs), equal Yin and Yang values (a zero
    sigma- plane) and an empty Yang patch."""
    import torch
    grid = small_yinyang(W, n_theta=13, n_phi=37, deg=4.0, n_r=67, l_max=9)
    rho = _special_density(grid, kind)
    with Plan(grid, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        got = phi.cpu().numpy()
    if kind == "zero":
        assert np.all(got == 0.0)
        return
    ref = oracle.solve(grid, rho)
    assert _rel_to_max(got, ref) <= TOL[precision], f"{kind} {precision}"


@pytest.mark.parametrize("precision", ["bf16x6", "fp16x3", "tf32x3"])
def test_signed_density_large_chunks(cuda, precision):
    """Signed density on a 2-degree grid with config-1 shells and degree
    (Nr = 400, l_max = 32), whose split-K chunks hold about 2000 cells: the
    field pass's monopole sums (FastTwoSum) run over long chunks of terms of
    both signs.  Zero-mean noise cancels: max |Phi(|rho|)| is ~400 x
    max |Phi(rho)| here, so the error is bounded normwise, as any rounded sum
    is, relative to the magnitudes summed (Phi of |rho|)."""
    import torch
    grid = small_yinyang(W, n_theta=46, n_phi=136, deg=2.0, n_r=400, l_max=32)
    rho = np.random.default_rng(9).standard_normal(grid.n_cells)
    ref = oracle.solve(grid, rho)
    scale = np.max(np.abs(oracle.solve(grid, np.abs(rho))))
    with Plan(grid, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        torch.cuda.synchronize()
        assert np.max(np.abs(phi.cpu().numpy() - ref)) <= TOL[precision] * scale
