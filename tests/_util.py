import math

import numpy as np


def rel_max(got, ref):
    """Largest elementwise relative error (ref must have no zeros)."""
    got = np.asarray(got); ref = np.asarray(ref)
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def rel_norm(got, ref):
    got = np.asarray(got); ref = np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


def col_rel(got, ref):
    """Per-column max error relative to the column's max magnitude."""
    got = np.asarray(got); ref = np.asarray(ref)
    scale = np.maximum(np.abs(ref).max(axis=0), 1e-300)
    return float(np.max(np.abs(got - ref).max(axis=0) / scale))


def small_yinyang(W, n_theta=6, n_phi=18, deg=8.0, n_r=9, l_max=6, **kw):
    return W.yinyang_grid(n_theta, n_phi, math.radians(deg), W.log_edges(n_r, 0.05), l_max, **kw)
