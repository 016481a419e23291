"""The non-orthogonal patches of Sect. 6 on the GPU: the cubed sphere (six
gnomonic cube faces, YGS_PATCH_GNOMONIC) with its weights U integrated
numerically on the device, against the oracle's own cell quadrature: the
weights, Phi in every precision, the moments, the adjoint and the uniform
sphere's closed form."""
import numpy as np
import pytest

import oracle
from paper_1903_08475_gb300 import Plan, ygs_backward, ygs_get_moments, ygs_get_weights, ygs_solve, workloads as W
from tests._util import col_rel, rel_max, rel_norm
from tests.test_oracle_pins import uniform_sphere, UNIFORM_EDGES

pytestmark = pytest.mark.gpu

GRIDS = {
    "cube_n6": lambda: W.cubed_sphere_grid(6, W.log_edges(9, 0.05), 7),
    "cube_ragged_rotated": lambda: W.cubed_sphere_grid(11, W.log_edges(23, 0.02), 9, G=1.7,
                                                       frame=(0.3, 1.1, -0.7)),
    "cube_centre_eval": lambda: W.cubed_sphere_grid(8, W.linear_edges(12, 0.1, 1.0), 12, eval=1),
}
TOL = {"fp64": 1e-12, "fp64tc": 1e-12, "fp64emu": 1e-12, "fp16x3": 1e-6, "bf16x6": 1e-6, "tf32x3": 1e-6}


@pytest.fixture(scope="module", params=sorted(GRIDS))
def case(request, cuda):
    g = GRIDS[request.param]()
    rho = W.random_density(g, 17)
    phi, B, M = oracle.solve(g, rho, moments=True)
    return request.param, g, rho, phi, B, M


def test_weights_match_oracle_quadrature(case):
    """U by the device's panel quadrature against the oracle's single-panel
    rule (two independent quadratures of the same integrals), Q at the
    evaluation points."""
    name, g, _, _, _, _ = case
    U_ref = oracle.build_U(g)
    Q_ref = oracle.build_Q(g)
    with Plan(g, "fp64") as plan:
        assert plan.info["symmetric"] == 0
        off = 0
        for p in range(g.n_patch):
            n = g.nang(p)
            U = ygs_get_weights(plan, "U", p)
            Q = ygs_get_weights(plan, "Q", p)
            assert np.abs(U - U_ref[off:off + n]).max() <= 1e-13 * np.abs(U_ref).max(), (name, p)
            assert np.abs(Q - Q_ref[off:off + n]).max() <= 1e-13 * abs(g.G), (name, p)
            off += n


@pytest.mark.parametrize("precision", sorted(TOL))
def test_phi_matches_oracle(case, precision):
    import torch
    name, g, rho, phi_ref, B_ref, M_ref = case
    with Plan(g, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda())
        B, M = ygs_get_moments(plan)
        torch.cuda.synchronize()
        assert rel_max(phi.cpu().numpy(), phi_ref) <= TOL[precision], (name, precision)
        if TOL[precision] <= 1e-12:
            assert col_rel(B.cpu().numpy(), B_ref) <= 1e-12
            assert col_rel(M.cpu().numpy(), M_ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp64emu"])
def test_adjoint_matches_oracle_transpose(case, precision):
    import torch
    name, g, rho, _, _, _ = case
    w = np.random.default_rng(3).standard_normal(g.n_cells)
    with Plan(g, precision) as plan:
        got = ygs_backward(plan, torch.from_numpy(w).cuda()).cpu().numpy()
    assert rel_norm(got, oracle.apply_T(g, w)) <= 1e-12, (name, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp64emu", "fp16x3"])
def test_uniform_sphere_closed_form(cuda, precision):
    """Only the monopole survives for a spherically symmetric density, so Phi
    at the shells' upper edges is the exact potential of the uniform ball."""
    import torch
    g = W.cubed_sphere_grid(9, UNIFORM_EDGES, 8, G=1.3, frame=(0.4, 0.9, 2.0))
    rho, exact = uniform_sphere(g)
    with Plan(g, precision) as plan:
        phi = ygs_solve(plan, torch.from_numpy(rho).cuda()).cpu().numpy()
    tol = 1e-12 if precision != "fp16x3" else 1e-6
    for p in range(g.n_patch):
        off, na = g.patch_offset(p), g.nang(p)
        ph = phi[off: off + g.n_r * na].reshape(g.n_r, na)
        assert np.abs(ph / exact[:, None] - 1).max() <= tol, (precision, p)
