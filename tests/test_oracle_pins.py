"""Pins of the CPU oracle against facts fixed outside it: values printed in
the paper, closed forms, textbook/library routines, invariants and brute
force.  No expected value here comes from the CUDA path."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_1903_08475_gb300 import workloads as W
from tests._util import rel_max, rel_norm, small_yinyang

GOLD = os.path.join(os.path.dirname(__file__), "golden", "yinyang_geometry.txt")


def golden():
    out = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        out[k] = np.array([float(x) for x in v])
    return out


def test_gauss_legendre_matches_numpy():
    for n in (1, 2, 5, 10, 17):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.abs(x - xr).max() < 1e-15 and np.abs(w - wr).max() < 1e-14


def test_euler_matrix_reproduces_printed_yin_yang_geometry():
    g = golden()
    Ryin = oracle.euler_matrix(*g["yin_euler"])
    assert np.abs(Ryin - g["yin_matrix"].reshape(3, 3)).max() < 1e-15
    Ryang = oracle.euler_matrix(*g["yang_euler"])
    # x = R_Yin xi_Yin and xi_Yin = M_YY xi_Yang  =>  R_Yang = R_Yin M_YY
    assert np.abs(Ryang - Ryin @ g["yy_matrix"].reshape(3, 3)).max() < 1e-15
    # the input generators' own rotation (scipy) agrees with the oracle's Eq. rottransmatrix
    rng = np.random.default_rng(0)
    for _ in range(5):
        e = rng.uniform(-3, 3, 3)
        assert np.abs(oracle.euler_matrix(*e) - W.rotation_matrix(*e)).max() < 1e-14


def test_real_harmonics_match_scipy():
    rng = np.random.default_rng(1)
    L = 20
    for _ in range(10):
        th, ph = rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi)
        Y = oracle.real_harmonics(L, th, ph)
        for l in range(L + 1):
            for m in range(l + 1):
                ycs = special.sph_harm_y(l, m, th, ph)  # normalised, Condon-Shortley phase
                f = (-1) ** m * math.sqrt(4 * math.pi / (2 * l + 1))
                if m == 0:
                    assert abs(Y[l * l] - f * ycs.real) < 1e-13
                else:
                    assert abs(Y[l * l + 2 * m - 1] - f * ycs.real) < 1e-13
                    assert abs(Y[l * l + 2 * m] - f * ycs.imag) < 1e-13


def test_addition_theorem_closed_form():
    rng = np.random.default_rng(2)
    L = 16
    for _ in range(10):
        a, b = rng.normal(size=3), rng.normal(size=3)
        a /= np.linalg.norm(a); b /= np.linalg.norm(b)
        ta, pa = math.acos(a[2]), math.atan2(a[1], a[0])
        tb, pb = math.acos(b[2]), math.atan2(b[1], b[0])
        Ya, Yb = oracle.real_harmonics(L, ta, pa), oracle.real_harmonics(L, tb, pb)
        for l in range(L + 1):
            s = sum((1.0 if m == 0 else 2.0) * (Ya[l * l + max(0, 2 * m - 1)] * Yb[l * l + max(0, 2 * m - 1)] +
                                                (Ya[l * l + 2 * m] * Yb[l * l + 2 * m] if m else 0.0))
                    for m in range(l + 1))
            assert abs(s - special.eval_legendre(l, a @ b)) < 1e-12


@pytest.mark.parametrize("l", [0, 1, 2, 3, 7, 30])
def test_radial_integrals_closed_form(l):
    for lo, hi in [(0.1, 0.2), (0.999, 1.0), (1e-3, 1.2e-3)]:
        rin = integrate.quad(lambda r: r ** (l + 2), lo, hi, epsabs=0, epsrel=1e-13)[0]
        rout = integrate.quad(lambda r: r ** (1 - l), lo, hi, epsabs=0, epsrel=1e-13)[0]
        assert abs(oracle.R_in(lo, hi, l) / rin - 1) < 1e-12
        assert abs(oracle.R_out(lo, hi, l) / rout - 1) < 1e-12
    assert abs(oracle.R_out(0.5, 1.0, 2) - math.log(2.0)) < 1e-15
    assert abs(oracle.R_in(0.0, 0.5, l) - 0.5 ** (l + 3) / (l + 3)) < 1e-16


def three_patch():
    rng = np.random.default_rng(5)
    eul = [W.random_euler(rng) for _ in range(3)]
    return W.make_grid(W.log_edges(5, 0.05), eul, [4, 3, 5], [7, 6, 5], [(0.3, 2.5), (0.6, 2.2), (0.0, math.pi)],
                       [(-2.0, 2.4), (-1.0, 1.7), (0.0, 2 * math.pi)], 5, G=1.7,
                       w=rng.uniform(0.2, 1.0, 4 * 7 + 3 * 6 + 5 * 5))


@pytest.mark.parametrize("make", [lambda: small_yinyang(W, n_theta=4, n_phi=10, n_r=5, l_max=5),
                                  lambda: W.polar_grid(5, 7, W.linear_edges(4, 0.2, 1.0), 4),
                                  three_patch,
                                  lambda: small_yinyang(W, n_theta=4, n_phi=10, n_r=4, l_max=4, eval=1),
                                  lambda: W.cubed_sphere_grid(4, W.linear_edges(4, 0.2, 1.0), 5),
                                  lambda: W.cubed_sphere_grid(3, W.log_edges(4, 0.05), 4, eval=1,
                                                              frame=(0.3, 1.1, -0.7))])
def test_three_oracle_routes_agree(make):
    """O1 (addition theorem with Legendre polynomials only) == O2 (global real
    harmonics) == O3 (per-patch superposition): three independent routes, on
    (theta, phi) patches and on the gnomonic cube faces of Sect. 6."""
    g = make()
    rho = W.random_density(g, 4)
    p2 = oracle.solve(g, rho)
    p1 = oracle.solve_direct(g, rho)
    p3 = oracle.solve_perpatch(g, rho)
    assert rel_max(p1, p2) < 1e-13
    assert rel_max(p3, p2) < 1e-13


UNIFORM_EDGES = np.array([0, 0.1, 0.2, 0.35, 0.5, 0.7, 0.9, 1.0])


def uniform_sphere(g, R=0.5, rho0=2.0):
    """Density rho0 in every cell of the shells inside radius R (a field layout
    [g][i][a]), and the exact potential at the upper shell edges r_i^+ (only
    the monopole survives: every l > 0 harmonic integrates to zero over the
    sphere)."""
    rho = np.zeros(g.n_cells)
    for p in range(g.n_patch):
        off, na = g.patch_offset(p), g.nang(p)
        for i in range(g.n_r):
            if g.edges[i + 1] <= R:
                rho[off + i * na: off + (i + 1) * na] = rho0
    r = g.edges[1:]
    exact = np.where(r >= R, -g.G * rho0 * (4 * np.pi / 3) * R ** 3 / r, -2 * np.pi * g.G * rho0 * (R ** 2 - r ** 2 / 3))
    return rho, exact


@pytest.mark.parametrize("make", [lambda: W.polar_grid(10, 20, UNIFORM_EDGES, 6, G=1.3),
                                  lambda: W.cubed_sphere_grid(6, UNIFORM_EDGES, 6, G=1.3, frame=(0.4, 0.9, 2.0))])
def test_uniform_sphere_exact(make):
    g = make()
    rho, exact = uniform_sphere(g)
    phi = oracle.solve(g, rho)
    for p in range(g.n_patch):
        off, na = g.patch_offset(p), g.nang(p)
        ph = phi[off: off + g.n_r * na].reshape(g.n_r, na)
        assert np.abs(ph / exact[:, None] - 1).max() < 1e-13


def test_cubed_sphere_tiles_the_sphere():
    """The six gnomonic faces (equiangular coordinates in [-pi/4, pi/4]^2,
    Sect. 6's non-orthogonal patches) cover the sphere once: the solid angles
    of all cells add to 4 pi, 4 pi / 6 per face, and every harmonic with l > 0
    integrates to zero over the union; the face centres are the six axes."""
    for frame in (None, (0.4, 0.9, 2.0)):
        g = W.cubed_sphere_grid(5, W.linear_edges(2, 0.5, 1.0), 6, frame=frame)
        U = oracle.build_U(g)  # U[a][0] = w * solid angle (Y_00 = 1)
        assert abs(U[:, 0].sum() - 4 * np.pi) < 1e-13
        na = g.nang(0)
        for p in range(6):
            assert abs(U[p * na:(p + 1) * na, 0].sum() - 4 * np.pi / 6) < 1e-13
        assert np.abs(U[:, 1:].sum(axis=0)).max() < 1e-13
    axes = sorted(tuple(np.round(W.rotation_matrix(*e) @ [0, 0, 1]).astype(int))
                  for e in W.cubed_sphere_grid(1, [0.5, 1.0], 0).euler)
    assert axes == sorted([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)])


def test_polar_grid_weights_are_separable_products():
    """N_g = 1, zero Euler angles: U = (2/delta_m) N_lm T_j {C_k, S_k}
    (Eqs. T_lm, C_k^m, S_k^m, a_ci/a_si), integrals done by scipy."""
    g = W.polar_grid(6, 8, W.linear_edges(2, 0.1, 1.0), 5)
    U = oracle.build_U(g)
    te = W.cell_edges_1d(0, math.pi, 6)
    pe = W.cell_edges_1d(0, 2 * math.pi, 8)
    for l in range(6):
        for m in range(l + 1):
            N = math.sqrt(math.factorial(l - m) / math.factorial(l + m))
            for j in range(6):
                T = integrate.quad(lambda t: math.sin(t) * special.lpmv(m, l, math.cos(t)) * (-1) ** m,
                                   te[j], te[j + 1], epsabs=1e-15, epsrel=1e-14)[0]
                for k in range(8):
                    C = (pe[k + 1] - pe[k]) if m == 0 else (math.sin(m * pe[k + 1]) - math.sin(m * pe[k])) / m
                    S = 0.0 if m == 0 else -(math.cos(m * pe[k + 1]) - math.cos(m * pe[k])) / m
                    f = 1.0 if m == 0 else 2.0
                    a = j * 8 + k
                    cC = l * l if m == 0 else l * l + 2 * m - 1
                    assert abs(U[a, cC] - f * N * T * C) < 1e-14
                    if m:
                        assert abs(U[a, l * l + 2 * m] - f * N * T * S) < 1e-14


def test_rotation_invariance():
    """Rotating every patch frame by the same R0 with the same local density
    leaves Phi on every local cell unchanged."""
    g = small_yinyang(W, n_theta=5, n_phi=14, n_r=6, l_max=8)
    rho = W.random_density(g, 9)
    frame = (0.4, 1.1, -2.3)
    g2 = W.yinyang_grid(5, 14, math.radians(8.0), W.log_edges(6, 0.05), 8, frame=frame)
    g2.w = g.w.copy()
    assert rel_max(oracle.solve(g2, rho), oracle.solve(g, rho)) < 1e-13


def test_quadrature_order_converged():
    for g in [small_yinyang(W), W.polar_grid(7, 13, W.linear_edges(3, 0.1, 1.0), 8), W.config0()[0],
              W.cubed_sphere_grid(6, W.linear_edges(2, 0.5, 1.0), 10), W.cubed_sphere_grid(16, [0.5, 1.0], 24)]:
        n = oracle.default_nq(g)
        U1 = oracle.build_U(g, nq=n)
        U2 = oracle.build_U(g, nq=n + 4)
        assert np.abs(U1 - U2).max() < 1e-15 * max(1.0, np.abs(U2).max()) * 10


def test_transpose_dot_product():
    g = small_yinyang(W, n_theta=4, n_phi=12, n_r=5, l_max=5)
    rho = W.random_density(g, 1)
    w = np.random.default_rng(2).standard_normal(g.n_cells)
    lhs = w @ oracle.solve(g, rho)
    rhs = oracle.apply_T(g, w) @ rho
    assert abs(lhs - rhs) < 1e-13 * np.abs(w).sum() * np.abs(oracle.solve(g, rho)).max()


def test_overlap_weights_cover_the_sphere():
    g = W.config0()[0]
    U = oracle.build_U(g)
    # column (0,0): w * solid angle, summed over both patches (Eq. A_lm_mult normalisation)
    assert abs(U[:, 0].sum() - 4 * math.pi) < 2e-3


class TestEllipsoid:
    def test_routes_agree(self):
        for (a, b, c) in [(0.6, 0.5, 0.4), (1.0, 1.5, 2.0)]:
            for X in [(0.1, 0.2, 0.05), (0.9, -0.3, 0.5), (0.3, 0.2, 2.5), (0.0, 0.0, 0.0)]:
                p1 = oracle.ellipsoid_phi(a, b, c, *X)[0]
                p2 = oracle.ellipsoid_phi(a, b, c, *X, route="paper")[0]
                assert abs(p1 - p2) < 1e-13 * abs(p1)

    def test_carlson_matches_scipy(self):
        for x, y, z in [(1, 2, 3), (0.3, 0.01, 5.0), (2, 2, 2)]:
            assert abs(oracle.carlson_rf(x, y, z) - special.elliprf(x, y, z)) < 1e-15
            assert abs(oracle.carlson_rd(x, y, z) - special.elliprd(x, y, z)) < 1e-14

    def test_sphere_limit_and_far_field(self):
        a = 0.7
        for r in [0.0, 0.3, 0.7, 1.5]:
            exact = -2 * np.pi * (a * a - r * r / 3) if r <= a else -(4 * np.pi / 3) * a ** 3 / r
            assert abs(oracle.ellipsoid_phi(a, a, a, r, 0, 0)[0] - exact) < 1e-13
        M = 4 * np.pi / 3 * 0.6 * 0.5 * 0.4
        far = oracle.ellipsoid_phi(0.6, 0.5, 0.4, 300.0, 200.0, 100.0)[0]
        assert abs(far * np.linalg.norm([300.0, 200.0, 100.0]) / (-M) - 1) < 1e-5

    def test_config0_discretisation_error(self):
        """Sect. 5.1 test at the small grid: error set by the surface
        representation (no exact gate exists; bounded here and recorded)."""
        g, rho = W.config0()
        phi = oracle.solve(g, rho)
        pts, vals = [], []
        idx = np.random.default_rng(0).choice(g.n_cells, 1500, replace=False)
        na = g.nang(0)
        for e in idx:
            p, rem = divmod(int(e), g.n_r * na)
            i, a = divmod(rem, na)
            j, k = divmod(a, g.n_phi[p])
            te = W.cell_edges_1d(*g.theta_range[p], g.n_theta[p])
            pe = W.cell_edges_1d(*g.phi_range[p], g.n_phi[p])
            d = W.local_dirs(te[j + 1], pe[k + 1]) @ W.rotation_matrix(*g.euler[p]).T
            pts.append(g.edges[i + 1] * d)
            vals.append(phi[e])
        pts = np.array(pts)
        ana = oracle.ellipsoid_phi(0.6, 0.5, 0.4, pts[:, 0], pts[:, 1], pts[:, 2])
        err = np.abs(np.array(vals) / ana - 1)
        assert err.max() < 5e-3 and np.median(err) < 2e-3


def test_point_mass_series_converges():
    """A small blob of mass at r0: outside it Phi tends to the truncated
    point-mass series -G m sum_l r0^l / r^(l+1) P_l(cos gamma) as the
    source cell shrinks (second order in the cell size)."""
    errs = []
    for n in (1, 2):
        nt, nf = 8 * n, 16 * n
        edges = np.concatenate([np.linspace(0.3, 0.32, 2 * n + 1), [0.5, 0.8, 1.0]])
        g = W.polar_grid(nt, nf, edges, 6)
        rho = np.zeros(g.n_cells)
        na = g.nang(0)
        # cells around theta ~ pi/2, phi ~ pi/8 inside shells of [0.3, 0.32]
        j0, k0 = nt // 2, nf // 16
        for i in range(2 * n):
            for j in range(j0, j0 + n):
                for k in range(k0, k0 + n):
                    rho[i * na + j * nf + k] = 1.0
        phi = oracle.solve(g, rho)
        # mass and centroid by direct integration of the cells
        te = W.cell_edges_1d(0, math.pi, nt); pe = W.cell_edges_1d(0, 2 * math.pi, nf)
        m = 0.0
        cen = np.zeros(3)
        for i in range(2 * n):
            vol_r = (edges[i + 1] ** 3 - edges[i] ** 3) / 3
            for j in range(j0, j0 + n):
                for k in range(k0, k0 + n):
                    dm = vol_r * (math.cos(te[j]) - math.cos(te[j + 1])) * (pe[k + 1] - pe[k])
                    c = W.local_dirs(0.5 * (te[j] + te[j + 1]), 0.5 * (pe[k] + pe[k + 1])) * 0.5 * (edges[i] + edges[i + 1])
                    m += dm
                    cen += dm * c
        cen /= m
        r0 = np.linalg.norm(cen)
        i_eval = len(edges) - 2  # r = 1.0
        a = (nt // 4) * nf + nf // 3
        d = W.local_dirs(te[a // nf + 1], pe[a % nf + 1])
        cg = d @ cen / r0
        series = -m * sum(r0 ** l * special.eval_legendre(l, cg) for l in range(7))
        errs.append(abs(phi[i_eval * na + a] / series - 1))
    assert errs[1] < errs[0] / 2.5 and errs[1] < 1e-3
