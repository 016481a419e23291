"""Seeded synthetic grids and densities for the multi-patch gravity solver.

This module builds INPUTS only: radial edges, patch extents and Euler angles,
the cell-constant overlap weights w_jk, and cell-averaged densities.  It holds
none of the solver's arithmetic (no spherical harmonics, no rotation of
harmonics, no radial moments); both the CUDA path and the CPU oracle consume
what it produces.  Its own geometry (local -> global directions) goes through
``scipy.spatial.transform.Rotation`` so that it shares no code with either.

Geometry conventions (arXiv:1903.08475):
  * patch-local spherical coordinates (theta, phi) with the Cartesian map of
    Eqs. cartosph-sphtocar; the global frame is x = R^(g) xi with R^(g) the
    z-y'-z'' Euler matrix of Eq. rottransmatrix, which equals the transpose of
    the active intrinsic rotation Rz(alpha) Ry(beta) Rz(gamma);
  * Yin-Yang patches span [pi/4 - d, 3pi/4 + d] x [-3pi/4 - d, 3pi/4 + d]
    (Sect. 4.1) with Euler angles (pi/2, pi/4, 3pi/2) for Yin and
    (pi/2, pi/4, pi/2) for Yang;
  * the overlap weight is the solid-angle average over each cell of 1/n_g,
    n_g the number of patches covering a direction (Eqs. A_lm_mult/B_lm_mult;
    the surface-averaged w_jk of Sect. 4.2);
  * fields are stored [patch][shell][theta][phi], phi fastest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
from scipy.spatial.transform import Rotation

SEED_BASE = 20190320

YIN_EULER = (math.pi / 2, math.pi / 4, 3 * math.pi / 2)
YANG_EULER = (math.pi / 2, math.pi / 4, math.pi / 2)


@dataclasses.dataclass
class Grid:
    """A multi-patch spherical grid (the ``ygs_desc`` of the C ABI)."""

    edges: np.ndarray            # (n_r + 1,) radial cell edges
    euler: np.ndarray            # (n_patch, 3) alpha, beta, gamma
    n_theta: np.ndarray          # (n_patch,) int
    n_phi: np.ndarray            # (n_patch,) int
    theta_range: np.ndarray      # (n_patch, 2)
    phi_range: np.ndarray        # (n_patch, 2)
    w: np.ndarray                # (sum n_theta*n_phi,) overlap weights
    l_max: int
    G: float = 1.0
    eval: int = 0                # 0 = upper vertex, 1 = angular centre
    kind: Optional[np.ndarray] = None  # (n_patch,) PATCH_LATLON / PATCH_GNOMONIC; None: all lat-lon

    @property
    def n_r(self) -> int:
        return len(self.edges) - 1

    @property
    def n_patch(self) -> int:
        return len(self.n_theta)

    def nang(self, p: int) -> int:
        return int(self.n_theta[p]) * int(self.n_phi[p])

    @property
    def nang_total(self) -> int:
        return sum(self.nang(p) for p in range(self.n_patch))

    @property
    def n_cells(self) -> int:
        return self.n_r * self.nang_total

    @property
    def K(self) -> int:
        return (self.l_max + 1) ** 2

    def patch_offset(self, p: int) -> int:
        """Element offset of patch p in a [g][i][a] field."""
        return self.n_r * sum(self.nang(q) for q in range(p))

    def with_lmax(self, l_max: int) -> "Grid":
        return dataclasses.replace(self, l_max=l_max)


# ------------------------------------------------------------------ geometry

def rotation_matrix(alpha: float, beta: float, gamma: float) -> np.ndarray:
    """x = R xi for the z-y'-z'' Euler angles of Eq. rottransmatrix."""
    return Rotation.from_euler("ZYZ", [alpha, beta, gamma]).as_matrix().T


def local_dirs(theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    st = np.sin(theta)
    return np.stack([st * np.cos(phi), st * np.sin(phi), np.cos(theta)], axis=-1)


def cell_edges_1d(lo: float, hi: float, n: int) -> np.ndarray:
    return lo + (hi - lo) * np.arange(n + 1) / n


def _gl(n: int):
    return np.polynomial.legendre.leggauss(n)


def _covered(grid_like, dirs_global: np.ndarray) -> np.ndarray:
    """Number of patches whose (theta, phi) extent contains each direction."""
    n = np.zeros(dirs_global.shape[:-1], dtype=np.int32)
    for p in range(len(grid_like["n_theta"])):
        R = rotation_matrix(*grid_like["euler"][p])
        loc = dirs_global @ R  # R^T x, row vectors
        th = np.arccos(np.clip(loc[..., 2], -1.0, 1.0))
        ph = np.arctan2(loc[..., 1], loc[..., 0])
        t0, t1 = grid_like["theta_range"][p]
        p0, p1 = grid_like["phi_range"][p]
        inside_t = (th >= t0 - 1e-13) & (th <= t1 + 1e-13)
        # azimuth: accept phi or phi +- 2 pi inside [p0, p1]
        inside_p = np.zeros_like(inside_t)
        for shift in (-2 * math.pi, 0.0, 2 * math.pi):
            inside_p |= (ph + shift >= p0 - 1e-13) & (ph + shift <= p1 + 1e-13)
        n += (inside_t & inside_p).astype(np.int32)
    return n


def _overlap_patch(gl, euler_p, tq, pq, wq_t, wq_p, nsub):
    """Cell averages of 1/n_g from the nsub x nsub sub-points given per cell."""
    nt, nf = tq.shape[0], pq.shape[0]
    TH = np.broadcast_to(tq[:, None, :, None], (nt, nf, nsub, nsub))
    PH = np.broadcast_to(pq[None, :, None, :], (nt, nf, nsub, nsub))
    glob = local_dirs(TH, PH) @ rotation_matrix(*euler_p).T
    ng = np.maximum(_covered(gl, glob), 1)
    W = wq_t[:, None, :, None] * wq_p[None, :, None, :]
    return (W / ng).sum(axis=(2, 3)) / W.sum(axis=(2, 3)), ng


def overlap_weights(euler, n_theta, n_phi, theta_range, phi_range, nsub: int = 16) -> np.ndarray:
    """Solid-angle average of 1/n_g over every cell (nsub x nsub Gauss-Legendre
    points).  Cells whose 4 x 4 probe points all see the same n_g take 1/n_g
    directly; the others are integrated with the full nsub x nsub rule."""
    gl = dict(euler=np.asarray(euler), n_theta=n_theta, theta_range=np.asarray(theta_range),
              phi_range=np.asarray(phi_range))
    out = []

    def nodes(edges, n):
        x, w = _gl(n)
        q = 0.5 * (edges[:-1, None] + edges[1:, None]) + 0.5 * (edges[1:, None] - edges[:-1, None]) * x[None, :]
        return q, w

    for p in range(len(n_theta)):
        te = cell_edges_1d(*theta_range[p], int(n_theta[p]))
        pe = cell_edges_1d(*phi_range[p], int(n_phi[p]))
        # probe pass: 4 x 4 points per cell
        tq, wt = nodes(te, 4)
        pq, wp = nodes(pe, 4)
        w4, ng4 = _overlap_patch(gl, euler[p], tq, pq, wt[None, :] * np.sin(tq), np.broadcast_to(wp, pq.shape), 4)
        uniform = (ng4.min(axis=(2, 3)) == ng4.max(axis=(2, 3)))
        w = np.where(uniform, 1.0 / ng4[:, :, 0, 0], 0.0)
        jj, kk = np.nonzero(~uniform)
        if len(jj):
            tq, wt = nodes(te, nsub)
            pq, wp = nodes(pe, nsub)
            for j0 in np.unique(jj):
                ks = kk[jj == j0]
                wsub, _ = _overlap_patch(gl, euler[p], tq[j0:j0 + 1], pq[ks], (wt * np.sin(tq[j0]))[None, :],
                                         np.broadcast_to(wp, (len(ks), nsub)), nsub)
                w[j0, ks] = wsub[0]
        out.append(w.reshape(-1))
    return np.concatenate(out)


def make_grid(edges, euler, n_theta, n_phi, theta_range, phi_range, l_max, G=1.0, eval=0, w=None,
              nsub_w: int = 16, kind=None) -> Grid:
    euler = np.asarray(euler, dtype=np.float64).reshape(-1, 3)
    n_theta = np.asarray(n_theta, dtype=np.int32).reshape(-1)
    n_phi = np.asarray(n_phi, dtype=np.int32).reshape(-1)
    theta_range = np.asarray(theta_range, dtype=np.float64).reshape(-1, 2)
    phi_range = np.asarray(phi_range, dtype=np.float64).reshape(-1, 2)
    if kind is not None:
        kind = np.asarray(kind, dtype=np.int32).reshape(-1)
        if w is None and np.any(kind != PATCH_LATLON):
            raise ValueError("overlap weights of gnomonic patches must be given")
    if w is None:
        w = overlap_weights(euler, n_theta, n_phi, theta_range, phi_range, nsub=nsub_w)
    return Grid(edges=np.asarray(edges, dtype=np.float64), euler=euler, n_theta=n_theta, n_phi=n_phi,
                theta_range=theta_range, phi_range=phi_range, w=np.asarray(w, dtype=np.float64),
                l_max=int(l_max), G=float(G), eval=int(eval), kind=kind)


def yinyang_extents(delta: float):
    return ((math.pi / 4 - delta, 3 * math.pi / 4 + delta), (-3 * math.pi / 4 - delta, 3 * math.pi / 4 + delta))


def yinyang_grid(n_theta: int, n_phi: int, delta: float, edges, l_max: int, G: float = 1.0, eval: int = 0,
                 frame=None, nsub_w: int = 16) -> Grid:
    """Yin-Yang pair; ``frame`` (3 Euler angles) optionally rotates the whole pair."""
    tr, pr = yinyang_extents(delta)
    eul = [YIN_EULER, YANG_EULER]
    if frame is not None:
        eul = [compose_euler(frame, e) for e in eul]
    return make_grid(edges, eul, [n_theta, n_theta], [n_phi, n_phi], [tr, tr], [pr, pr], l_max, G, eval,
                     nsub_w=nsub_w)


def yinyang_resolution(deg: float):
    """Cells per patch for an angular resolution of ``deg`` degrees with a
    one-cell extension on each side (d = resolution), as in Sect. 4.1."""
    d = math.radians(deg)
    n_theta = int(round((math.pi / 2 + 2 * d) / d))
    n_phi = int(round((3 * math.pi / 2 + 2 * d) / d))
    return n_theta, n_phi, d


def polar_grid(n_theta: int, n_phi: int, edges, l_max: int, G: float = 1.0, eval: int = 0) -> Grid:
    """The single spherical polar patch (N_g = 1, zero Euler angles, w = 1)."""
    return make_grid(edges, [(0.0, 0.0, 0.0)], [n_theta], [n_phi], [(0.0, math.pi)], [(0.0, 2 * math.pi)],
                     l_max, G, eval, w=np.ones(n_theta * n_phi))


PATCH_LATLON, PATCH_GNOMONIC = 0, 1


def euler_from_matrix(R) -> tuple:
    """Euler angles (alpha, beta, gamma) with rotation_matrix(alpha, beta, gamma) = R."""
    R = np.asarray(R, dtype=np.float64)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")  # gimbal lock at beta = 0 or pi: any split of alpha + gamma will do
        ang = Rotation.from_matrix(R.T).as_euler("ZYZ")
    if not np.allclose(rotation_matrix(*ang), R, atol=1e-12):
        raise ValueError("not a rotation matrix")
    return tuple(float(x) for x in ang)


# The six faces of the cube as rotations x = R v of a face's local frame
# (local z = the face normal; local x, y along cube edges, right-handed).
CUBE_FACES = (
    np.eye(3),                                                     # +z
    np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], dtype=float),    # -z
    np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]], dtype=float),      # +x: x -> +y, y -> +z, z -> +x
    np.array([[0, 0, -1], [-1, 0, 0], [0, 1, 0]], dtype=float),    # -x
    np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=float),      # +y: x -> +z, y -> +x, z -> +y
    np.array([[0, 1, 0], [0, 0, -1], [-1, 0, 0]], dtype=float),    # -y
)


def cubed_sphere_grid(n: int, edges, l_max: int, G: float = 1.0, eval: int = 0, frame=None) -> Grid:
    """The cubed sphere (the non-orthogonal patches of Sect. 6): six gnomonic
    faces, each n x n cells in the equiangular coordinates (xi, eta) in
    [-pi/4, pi/4]^2; the faces tile the sphere, so every overlap weight is 1.
    ``frame`` (3 Euler angles) optionally rotates the whole cube."""
    eul = [euler_from_matrix(R) for R in CUBE_FACES]
    if frame is not None:
        eul = [compose_euler(frame, e) for e in eul]
    q = math.pi / 4
    return make_grid(edges, eul, [n] * 6, [n] * 6, [(-q, q)] * 6, [(-q, q)] * 6, l_max, G, eval,
                     w=np.ones(6 * n * n), kind=[PATCH_GNOMONIC] * 6)


def compose_euler(outer, inner):
    """Euler angles of the frame x = R(outer) R(inner) xi."""
    R = rotation_matrix(*outer) @ rotation_matrix(*inner)
    act = Rotation.from_matrix(R.T)
    a, b, g = act.as_euler("ZYZ")
    return (float(a), float(b), float(g))


def log_edges(n_r: int, r_min: float, r_max: float = 1.0) -> np.ndarray:
    """edges[0] = 0, edges[1..n_r] log-spaced in [r_min, r_max]: the innermost
    shell is the ball of radius r_min."""
    return np.concatenate([[0.0], np.geomspace(r_min, r_max, n_r)])


def linear_edges(n_r: int, r_in: float, r_out: float) -> np.ndarray:
    return np.linspace(r_in, r_out, n_r + 1)


# ---------------------------------------------------------------- densities

def _sub_points(grid: Grid, p: int, nsub: int):
    """Equal-volume sub-cell centres: radii (n_r, nsub) uniform in r^3, and
    global directions (nang, nsub*nsub, 3) uniform in cos(theta) and phi."""
    e = grid.edges
    u = (np.arange(nsub) + 0.5) / nsub
    r3 = e[:-1, None] ** 3 + (e[1:, None] ** 3 - e[:-1, None] ** 3) * u[None, :]
    radii = np.cbrt(r3)
    te = cell_edges_1d(*grid.theta_range[p], int(grid.n_theta[p]))
    pe = cell_edges_1d(*grid.phi_range[p], int(grid.n_phi[p]))
    ct = np.cos(te[:-1, None]) + (np.cos(te[1:, None]) - np.cos(te[:-1, None])) * u[None, :]
    th = np.arccos(np.clip(ct, -1, 1))                               # (nt, nsub)
    ph = pe[:-1, None] + (pe[1:, None] - pe[:-1, None]) * u[None, :]  # (nf, nsub)
    nt, nf = th.shape[0], ph.shape[0]
    TH = np.broadcast_to(th[:, None, :, None], (nt, nf, nsub, nsub))
    PH = np.broadcast_to(ph[None, :, None, :], (nt, nf, nsub, nsub))
    loc = local_dirs(TH, PH).reshape(nt * nf, nsub * nsub, 3)
    glob = loc @ rotation_matrix(*grid.euler[p]).T
    return radii, glob


def ellipsoid_density(grid: Grid, axes=(0.6, 0.5, 0.4), body_rot=None, rho0: float = 1.0, nsub: int = 4) -> np.ndarray:
    """Cell volume fraction of a homogeneous ellipsoid (nsub^3 equal-volume
    sub-cells) times rho0.  ``body_rot`` is a 3x3 matrix mapping body-frame
    coordinates to global ones (None: axes along global x, y, z)."""
    a = np.asarray(axes, dtype=np.float64)
    Rb = np.eye(3) if body_rot is None else np.asarray(body_rot)
    out = np.empty(grid.n_cells)
    nr = grid.n_r
    for p in range(grid.n_patch):
        radii, dirs = _sub_points(grid, p, nsub)
        na = dirs.shape[0]
        body = dirs @ Rb
        Rsurf = 1.0 / np.sqrt(((body / a) ** 2).sum(-1))               # (nang, nsub^2)
        # number of radial sub-points (all shells, ascending) inside along each direction
        n_in = np.searchsorted(radii.reshape(-1), Rsurf.reshape(-1), side="right").reshape(na, -1)
        full, part = np.divmod(n_in, nsub)                              # shells fully inside, remainder
        cnt = np.zeros((nr + 2, na))
        aa = np.broadcast_to(np.arange(na)[:, None], full.shape)
        np.add.at(cnt, (np.minimum(full, nr + 1).ravel(), aa.ravel()), 1.0)
        inside = cnt[::-1].cumsum(axis=0)[::-1]                         # #dirs with full >= k
        frac = nsub * inside[1:nr + 1]                                  # shells i < full
        pw = np.zeros((nr + 1, na))
        np.add.at(pw, (np.minimum(full, nr).ravel(), aa.ravel()), part.ravel().astype(np.float64))
        frac += pw[:nr]
        frac /= nsub * dirs.shape[1]
        off = grid.patch_offset(p)
        out[off: off + nr * na] = (rho0 * frac).reshape(-1)
    return out


def gaussian_blobs_density(grid: Grid, centres, sigma: float = 0.05, amplitude: float = 5.0, nsub: int = 4) -> np.ndarray:
    """Cell average (nsub^3 sub-cells) of sum_b A exp(-|x - c_b|^2 / (2 sigma^2));
    cells farther than 8.5 sigma (exp(-36)) from a centre get no contribution."""
    out = np.zeros(grid.n_cells)
    nr = grid.n_r
    cut = sigma * math.sqrt(72.0)
    for p in range(grid.n_patch):
        radii, dirs = _sub_points(grid, p, nsub)
        na = dirs.shape[0]
        cdir = dirs.mean(axis=1)
        cdir /= np.linalg.norm(cdir, axis=1, keepdims=True)
        ang_rad = np.arccos(np.clip((dirs * cdir[:, None, :]).sum(-1).min(1), -1, 1))  # angular half-size
        blk = np.zeros((nr, na))
        for c in np.asarray(centres, dtype=np.float64).reshape(-1, 3):
            rc = float(np.linalg.norm(c))
            chat = c / max(rc, 1e-300)
            gam = np.arccos(np.clip(cdir @ chat, -1, 1))
            for i in range(nr):
                r0, r1 = grid.edges[i], grid.edges[i + 1]
                if r1 < rc - cut or r0 > rc + cut:
                    continue
                # lower bound of the distance between the blob centre and cells of shell i
                gmin = np.maximum(gam - ang_rad, 0.0)
                rr = np.clip(rc * np.cos(np.minimum(gmin, math.pi / 2)), r0, r1)
                dmin2 = rr * rr - 2 * rr * rc * np.cos(gmin) + rc * rc
                sel = np.nonzero(dmin2 <= cut * cut)[0]
                if len(sel) == 0:
                    continue
                dc = dirs[sel] @ c                                   # (ns, s2) = rc cos
                acc = np.zeros(len(sel))
                for s_ in range(radii.shape[1]):
                    r = radii[i, s_]
                    d2 = r * r - 2 * r * dc + rc * rc
                    acc += np.exp(-d2 / (2 * sigma * sigma)).mean(1)
                blk[i, sel] += amplitude * acc / radii.shape[1]
        off = grid.patch_offset(p)
        out[off: off + nr * na] = blk.reshape(-1)
    return out


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    return Rotation.random(random_state=rng).as_matrix()


def random_euler(rng: np.random.Generator):
    a, b, g = Rotation.random(random_state=rng).as_euler("ZYZ")
    return (float(a), float(b), float(g))


def lognormal_density(grid: Grid, rng: np.random.Generator, n_fft: int = 256, sigma_ln: float = 0.5,
                      r_core: float = 0.05) -> np.ndarray:
    """exp(s g - s^2/2) (1 + (r/r_core)^2)^-1.5 with g a unit-variance Gaussian
    random field of power spectrum k^-2 on an n_fft^3 grid over [-1,1]^3,
    sampled trilinearly at cell centres."""
    white = rng.standard_normal((n_fft,) * 3)
    f = np.fft.rfftn(white)
    k1 = np.fft.fftfreq(n_fft) * n_fft
    k3 = np.fft.rfftfreq(n_fft) * n_fft
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k3[None, None, :] ** 2)
    amp = np.zeros_like(kk)
    amp[kk > 0] = 1.0 / kk[kk > 0]
    g = np.fft.irfftn(f * amp, s=(n_fft,) * 3)
    g = (g - g.mean()) / g.std()
    out = np.empty(grid.n_cells)
    e = grid.edges
    rc = 0.5 * (e[:-1] + e[1:])
    for p in range(grid.n_patch):
        te = cell_edges_1d(*grid.theta_range[p], int(grid.n_theta[p]))
        pe = cell_edges_1d(*grid.phi_range[p], int(grid.n_phi[p]))
        th = 0.5 * (te[:-1] + te[1:])
        ph = 0.5 * (pe[:-1] + pe[1:])
        TH, PH = np.meshgrid(th, ph, indexing="ij")
        d = (local_dirs(TH, PH).reshape(-1, 3)) @ rotation_matrix(*grid.euler[p]).T
        off = grid.patch_offset(p)
        na = grid.nang(p)
        for i in range(grid.n_r):
            x = rc[i] * d
            u = (x + 1.0) * 0.5 * (n_fft - 1)
            i0 = np.clip(np.floor(u).astype(np.int64), 0, n_fft - 2)
            t = np.clip(u - i0, 0.0, 1.0)
            val = np.zeros(na)
            for dx in (0, 1):
                for dy in (0, 1):
                    for dz in (0, 1):
                        wgt = ((t[:, 0] if dx else 1 - t[:, 0]) * (t[:, 1] if dy else 1 - t[:, 1]) *
                               (t[:, 2] if dz else 1 - t[:, 2]))
                        val += wgt * g[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
            prof = (1.0 + (rc[i] / r_core) ** 2) ** -1.5
            out[off + i * na: off + (i + 1) * na] = np.exp(sigma_ln * val - 0.5 * sigma_ln ** 2) * prof
    return out


# ------------------------------------------------------------- the configs

def config0(l_max: int = 12, nsub_w: int = 16):
    """Yin-Yang, Nr = 64 log-spaced shells in [0.01, 1], 24 x 72 cells per
    patch (overlap of two theta cells), l_max = 12, G = 1; density 1 inside
    the ellipsoid (0.6, 0.5, 0.4) with axes along global x, y, z."""
    n_theta, n_phi = 24, 72
    dth = (math.pi / 2) / (n_theta - 4)  # pi/2 + 4 dth = 24 dth
    delta = 2 * dth
    grid = yinyang_grid(n_theta, n_phi, delta, log_edges(64, 0.01, 1.0), l_max, nsub_w=nsub_w)
    rho = ellipsoid_density(grid, (0.6, 0.5, 0.4))
    return grid, rho


def config1_grid(n_r: int = 400, deg: float = 1.0, l_max: int = 32, r_min: float = 1e-3, nsub_w: int = 16) -> Grid:
    n_theta, n_phi, d = yinyang_resolution(deg)
    return yinyang_grid(n_theta, n_phi, d, log_edges(n_r, r_min, 1.0), l_max, nsub_w=nsub_w)


def config1_density(grid: Grid, seed: int = SEED_BASE + 1) -> np.ndarray:
    """Ellipsoid (0.6, 0.5, 0.4) rotated by seeded Euler angles plus three
    Gaussian blobs (sigma 0.05, amplitude 5) centred uniformly in r < 0.7."""
    rng = np.random.default_rng(seed)
    Rb = random_rotation(rng)
    rho = ellipsoid_density(grid, (0.6, 0.5, 0.4), body_rot=Rb)
    centres = []
    while len(centres) < 3:
        c = rng.uniform(-0.7, 0.7, 3)
        if np.linalg.norm(c) < 0.7:
            centres.append(c)
    rho += gaussian_blobs_density(grid, centres)
    return rho


def _cache_path(tag: str) -> str:
    import hashlib
    import os
    import tempfile
    d = os.environ.get("YGS_INPUT_CACHE") or os.path.join(tempfile.gettempdir(), "ygs_inputs")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, hashlib.sha1(tag.encode()).hexdigest()[:20] + ".npy")


def cached(tag: str, make):
    """Memoises an input array on local disk (a temporary directory) by tag."""
    import os
    path = _cache_path(tag)
    if os.path.exists(path):
        try:
            return np.load(path)
        except Exception:
            pass
    arr = make()
    tmp = path + f".{os.getpid()}.npy"
    np.save(tmp, arr)
    os.replace(tmp, path)
    return arr


def config1(seed: int = SEED_BASE + 1, **kw):
    grid = config1_grid(**kw)
    tag = f"cfg1-density-v1-{seed}-{sorted(kw.items())}"
    return grid, cached(tag, lambda: config1_density(grid, seed))


def config2(seed: int = SEED_BASE + 2, n_fft: int = 256):
    # 0.5 degree cells with a two-cell (1 degree) extension on each side
    n_theta, n_phi, d = 184, 544, math.radians(1.0)
    grid = yinyang_grid(n_theta, n_phi, d, log_edges(800, 1e-3, 1.0), 64)
    rng = np.random.default_rng(seed)
    return grid, lognormal_density(grid, rng, n_fft=n_fft)


def config4(seed: int = SEED_BASE + 4):
    """Adjoint workload: Yin-Yang 1 degree, Nr = 256, l_max = 32, the config-1
    density, and seeded N(0, 1) weights w of J = sum_cells w Phi(rho)."""
    grid = config1_grid(n_r=256)
    tag = f"cfg4-density-v1-{seed}"
    rho = cached(tag, lambda: config1_density(grid, SEED_BASE + 1))
    w = np.random.default_rng(seed).standard_normal(grid.n_cells)
    return grid, rho, w


def random_density(grid: Grid, seed: int) -> np.ndarray:
    """Positive random density, uniform in [0.5, 1.5) (for parity cases)."""
    return np.random.default_rng(seed).uniform(0.5, 1.5, grid.n_cells)


# ------------------------------------------------------- config 3 (batches)

def six_patch_grid(n_theta: int, n_phi: int, delta: float, edges, l_max: int, frames, w=None,
                   nsub_w: int = 8) -> Grid:
    """Three Yin-Yang pairs, pair q rotated as a whole by the Euler angles
    frames[q]: six patches covering every direction three times."""
    tr, pr = yinyang_extents(delta)
    eul = [compose_euler(f, e) for f in frames for e in (YIN_EULER, YANG_EULER)]
    return make_grid(edges, eul, [n_theta] * 6, [n_phi] * 6, [tr] * 6, [pr] * 6, l_max, w=w, nsub_w=nsub_w)


def config3(n_fields: int = 64, seed: int = SEED_BASE + 3):
    """A batch of uneven fields: Nr uniform in [128, 600] (log-spaced shells
    in [1e-3, 1]), resolution 2, 1.5 or 1 degree, l_max uniform in [16, 48],
    patch set Yin-Yang or six patches (three rotated Yin-Yang pairs drawn from a
    pool of four; six-patch sets at 2 and 1.5 degrees only), densities
    alternating between the config-1 kind (rotated ellipsoid plus three
    blobs) and the config-2 kind (lognormal times a central profile), both
    sampled at cell centres (see batch_density).  Overlap weights depend only on
    the angular layout, so they are computed once per (patch set, resolution)
    and shared.  Returns a list of (grid, density kind, density seed)."""
    rng = np.random.default_rng(seed)
    frames_pool = [[random_euler(rng) for _ in range(3)] for _ in range(4)]
    w_pool = {}
    out = []
    for k in range(n_fields):
        n_r = int(rng.integers(128, 601))
        deg = float(rng.choice([2.0, 1.5, 1.0]))
        l_max = int(rng.integers(16, 49))
        six = bool(rng.random() < 0.5) and deg != 1.0
        pick = int(rng.integers(0, 4))
        nt, nf, d = yinyang_resolution(deg)
        edges = log_edges(n_r, 1e-3, 1.0)
        key = (deg, pick if six else -1)
        if key not in w_pool:
            g0 = (six_patch_grid(nt, nf, d, edges[:2], 0, frames_pool[pick]) if six
                  else yinyang_grid(nt, nf, d, edges[:2], 0, nsub_w=8))
            w_pool[key] = g0.w
        if six:
            grid = six_patch_grid(nt, nf, d, edges, l_max, frames_pool[pick], w=w_pool[key])
        else:
            tr, pr = yinyang_extents(d)
            grid = make_grid(edges, [YIN_EULER, YANG_EULER], [nt, nt], [nf, nf], [tr, tr], [pr, pr], l_max,
                             w=w_pool[key])
        out.append((grid, "blobs" if k % 2 == 0 else "lognormal", seed * 1000 + k))
    return out


def batch_density(grid: Grid, kind: str, seed: int, device="cpu"):
    """Density of a config-3 field at cell centres as a torch FP64 tensor on
    ``device`` (fast enough for tens of millions of cells on a GPU).
    "blobs": 1 inside the ellipsoid (0.6, 0.5, 0.4) rotated by seeded Euler
    angles plus three Gaussian blobs (sigma 0.05, amplitude 5, centres in
    r < 0.7).  "lognormal": exp(0.5 g - 0.125) (1 + (r/0.05)^2)^-1.5 with g a
    unit-variance sum of 32 random Fourier modes, amplitudes ~ 1/k (power
    spectrum k^-2) for wavenumbers pi .. 16 pi."""
    import torch
    rng = np.random.default_rng(seed)
    e = grid.edges
    rc = torch.tensor(0.5 * (e[:-1] + e[1:]), dtype=torch.float64, device=device)
    if kind == "blobs":
        Rb = random_rotation(rng)
        ax = np.array([0.6, 0.5, 0.4])
        centres = []
        while len(centres) < 3:
            c = rng.uniform(-0.7, 0.7, 3)
            if np.linalg.norm(c) < 0.7:
                centres.append(c)
    else:
        kdir = rng.standard_normal((32, 3))
        kdir /= np.linalg.norm(kdir, axis=1, keepdims=True)
        kmag = np.pi * np.exp(rng.uniform(0.0, np.log(16.0), 32))
        kv = torch.tensor(kdir * kmag[:, None], dtype=torch.float64, device=device)
        amp = torch.tensor(1.0 / kmag, dtype=torch.float64, device=device)
        amp = amp / torch.sqrt(0.5 * (amp * amp).sum())
        phase = torch.tensor(rng.uniform(0, 2 * np.pi, 32), dtype=torch.float64, device=device)
    parts = []
    for p in range(grid.n_patch):
        te = cell_edges_1d(*grid.theta_range[p], int(grid.n_theta[p]))
        pe = cell_edges_1d(*grid.phi_range[p], int(grid.n_phi[p]))
        TH, PH = np.meshgrid(0.5 * (te[:-1] + te[1:]), 0.5 * (pe[:-1] + pe[1:]), indexing="ij")
        d = local_dirs(TH, PH).reshape(-1, 3) @ rotation_matrix(*grid.euler[p]).T
        if kind == "blobs":
            db = torch.tensor(d @ Rb, dtype=torch.float64, device=device)     # body-frame directions
            q = ((db / torch.tensor(ax, dtype=torch.float64, device=device)) ** 2).sum(1)
            rho = ((rc[:, None] ** 2) * q[None, :] <= 1.0).to(torch.float64)
            dg = torch.tensor(d, dtype=torch.float64, device=device)
            for c in centres:
                ct = torch.tensor(c, dtype=torch.float64, device=device)
                d2 = rc[:, None] ** 2 - 2 * rc[:, None] * (dg @ ct)[None, :] + float(c @ c)
                rho += 5.0 * torch.exp(-d2 / (2 * 0.05 ** 2))
        else:
            dg = torch.tensor(d, dtype=torch.float64, device=device)
            kd = dg @ kv.T                                                   # (na, 32)
            g = torch.zeros(len(rc), dg.shape[0], dtype=torch.float64, device=device)
            for m in range(32):
                g += amp[m] * torch.cos(rc[:, None] * kd[None, :, m] + phase[m])
            prof = (1.0 + (rc / 0.05) ** 2) ** -1.5
            rho = torch.exp(0.5 * g - 0.125) * prof[:, None]
        parts.append(rho.reshape(-1))
    return torch.cat(parts)


def config2_grid() -> Grid:
    """The config-2 grid (0.5 degree Yin-Yang, Nr = 800, l_max = 64) alone."""
    return yinyang_grid(184, 544, math.radians(1.0), log_edges(800, 1e-3, 1.0), 64)


def lognormal_density_torch(grid: Grid, seed: int = SEED_BASE + 2, n_fft: int = 256, sigma_ln: float = 0.5,
                            r_core: float = 0.05, device="cpu"):
    """lognormal_density computed with torch on ``device`` (the same recipe: a
    unit-variance k^-2 Gaussian field from a seeded n_fft^3 FFT on [-1,1]^3,
    sampled trilinearly at cell centres, exp(s g - s^2/2) (1 + (r/r_core)^2)^-1.5),
    for grids of 1e8 cells.  Returns an FP64 tensor."""
    import torch
    rng = np.random.default_rng(seed)
    white = torch.from_numpy(rng.standard_normal((n_fft,) * 3)).to(device)
    f = torch.fft.rfftn(white)
    k1 = torch.fft.fftfreq(n_fft, device=device, dtype=torch.float64) * n_fft
    k3 = torch.fft.rfftfreq(n_fft, device=device, dtype=torch.float64) * n_fft
    kk = torch.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k3[None, None, :] ** 2)
    amp = torch.where(kk > 0, 1.0 / torch.clamp(kk, min=1e-300), torch.zeros_like(kk))
    g = torch.fft.irfftn(f * amp, s=(n_fft,) * 3)
    g = (g - g.mean()) / g.std(correction=0)
    e = grid.edges
    rc = torch.tensor(0.5 * (e[:-1] + e[1:]), dtype=torch.float64, device=device)
    parts = []
    for p in range(grid.n_patch):
        te = cell_edges_1d(*grid.theta_range[p], int(grid.n_theta[p]))
        pe = cell_edges_1d(*grid.phi_range[p], int(grid.n_phi[p]))
        TH, PH = np.meshgrid(0.5 * (te[:-1] + te[1:]), 0.5 * (pe[:-1] + pe[1:]), indexing="ij")
        d = torch.tensor(local_dirs(TH, PH).reshape(-1, 3) @ rotation_matrix(*grid.euler[p]).T,
                         dtype=torch.float64, device=device)
        out = torch.empty(grid.n_r, d.shape[0], dtype=torch.float64, device=device)
        for i in range(grid.n_r):
            u = (rc[i] * d + 1.0) * 0.5 * (n_fft - 1)
            i0 = torch.clamp(torch.floor(u).long(), 0, n_fft - 2)
            t = torch.clamp(u - i0, 0.0, 1.0)
            val = torch.zeros(d.shape[0], dtype=torch.float64, device=device)
            for dx in (0, 1):
                for dy in (0, 1):
                    for dz in (0, 1):
                        wgt = ((t[:, 0] if dx else 1 - t[:, 0]) * (t[:, 1] if dy else 1 - t[:, 1]) *
                               (t[:, 2] if dz else 1 - t[:, 2]))
                        val += wgt * g[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
            prof = (1.0 + (rc[i] / r_core) ** 2) ** -1.5
            out[i] = torch.exp(sigma_ln * val - 0.5 * sigma_ln ** 2) * prof
        parts.append(out.reshape(-1))
    return torch.cat(parts)
