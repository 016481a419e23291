"""Input generators: the torch lognormal field (used for the full-size
0.5-degree bench) equals the numpy one of the parity tests, and the config-3
batch has the stated distribution."""
import math

import numpy as np
import pytest

from paper_1903_08475_gb300 import workloads as W


def test_lognormal_torch_matches_numpy():
    g = W.yinyang_grid(12, 34, math.radians(8.0), W.log_edges(6, 1e-2, 1.0), 4)
    a = W.lognormal_density(g, np.random.default_rng(7), n_fft=32)
    b = W.lognormal_density_torch(g, seed=7, n_fft=32).numpy()
    assert np.max(np.abs(a - b) / np.abs(a)) <= 1e-12


def test_config3_distribution():
    fields = W.config3(n_fields=12)
    assert len(fields) == 12
    for grid, kind, seed in fields:
        assert 128 <= grid.n_r <= 600 and 16 <= grid.l_max <= 48
        assert grid.n_patch in (2, 6) and kind in ("blobs", "lognormal")
        # overlap weights cover the sphere once: sum w dOmega = 4 pi
        tot = 0.0
        for p in range(grid.n_patch):
            te = W.cell_edges_1d(*grid.theta_range[p], int(grid.n_theta[p]))
            pe = W.cell_edges_1d(*grid.phi_range[p], int(grid.n_phi[p]))
            dom = np.outer(np.cos(te[:-1]) - np.cos(te[1:]), np.diff(pe)).reshape(-1)
            off = sum(grid.nang(q) for q in range(p))
            tot += float(dom @ grid.w[off:off + grid.nang(p)])
        assert abs(tot - 4 * math.pi) <= 2e-3 * 4 * math.pi
    rho = W.batch_density(fields[0][0], fields[0][1], fields[0][2])
    assert rho.shape[0] == fields[0][0].n_cells and float(rho.min()) >= 0.0
