"""CPU FP64 oracle for the multi-patch gravity solver -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
library never does: it shares no code with the CUDA path.  The arithmetic
lives in ``ygs_oracle.c`` (plain C, FP64, OpenMP); this module compiles it
with gcc on first use and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ygs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libygs_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _Grid(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("edges", _dp), ("n_patch", ctypes.c_int), ("euler", _dp),
                ("n_theta", _ip), ("n_phi", _ip), ("theta_range", _dp), ("phi_range", _dp),
                ("w", _dp), ("l_max", ctypes.c_int), ("G", ctypes.c_double), ("eval", ctypes.c_int),
                ("kind", _ip)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.ora_ellipsoid_phi.restype = ctypes.c_double
            L.ora_ellipsoid_phi_paper.restype = ctypes.c_double
            L.ora_carlson_rf.restype = ctypes.c_double
            L.ora_carlson_rd.restype = ctypes.c_double
            L.ora_R_in.restype = ctypes.c_double
            L.ora_R_out.restype = ctypes.c_double
            for f in ("ora_ellipsoid_phi", "ora_ellipsoid_phi_paper"):
                getattr(L, f).argtypes = [ctypes.c_double] * 8
            L.ora_carlson_rf.argtypes = [ctypes.c_double] * 3
            L.ora_carlson_rd.argtypes = [ctypes.c_double] * 3
            L.ora_R_in.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
            L.ora_R_out.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


class _Keep:
    pass


def _grid(g):
    k = _Keep()
    k.edges = np.ascontiguousarray(g.edges, dtype=np.float64)
    k.euler = np.ascontiguousarray(g.euler, dtype=np.float64).reshape(-1)
    k.nt = np.ascontiguousarray(g.n_theta, dtype=np.int32)
    k.nf = np.ascontiguousarray(g.n_phi, dtype=np.int32)
    k.tr = np.ascontiguousarray(g.theta_range, dtype=np.float64).reshape(-1)
    k.pr = np.ascontiguousarray(g.phi_range, dtype=np.float64).reshape(-1)
    k.w = np.ascontiguousarray(g.w, dtype=np.float64)
    kind = getattr(g, "kind", None)
    k.kind = None if kind is None else np.ascontiguousarray(kind, dtype=np.int32)
    s = _Grid(g.n_r, _p(k.edges), g.n_patch, _p(k.euler), k.nt.ctypes.data_as(_ip), k.nf.ctypes.data_as(_ip),
              _p(k.tr), _p(k.pr), _p(k.w), g.l_max, g.G, g.eval,
              None if k.kind is None else k.kind.ctypes.data_as(_ip))
    k.s = s
    return k


def default_nq(g) -> int:
    """Quadrature order per cell direction: enough nodes for l_max x cell width."""
    h = 0.0
    for p in range(g.n_patch):
        h = max(h, (g.theta_range[p][1] - g.theta_range[p][0]) / g.n_theta[p],
                (g.phi_range[p][1] - g.phi_range[p][0]) / g.n_phi[p])
    return int(6 + np.ceil(1.2 * (g.l_max + 2) * h))


def num_threads() -> int:
    return lib().ora_num_threads()


def gauss_legendre(n: int):
    x = np.empty(n); w = np.empty(n)
    lib().ora_gauss_legendre(n, _p(x), _p(w))
    return x, w


def euler_matrix(alpha, beta, gamma):
    R = np.empty(9)
    lib().ora_euler_matrix(ctypes.c_double(alpha), ctypes.c_double(beta), ctypes.c_double(gamma), _p(R))
    return R.reshape(3, 3)


def real_harmonics(l_max, theta, phi):
    out = np.empty((l_max + 1) ** 2)
    lib().ora_real_harmonics(l_max, ctypes.c_double(theta), ctypes.c_double(phi), _p(out))
    return out


def R_in(lo, hi, l):
    return lib().ora_R_in(lo, hi, l)


def R_out(lo, hi, l):
    return lib().ora_R_out(lo, hi, l)


def build_U(g, nq=None, local=False):
    k = _grid(g)
    U = np.empty((g.nang_total, g.K))
    f = lib().ora_build_U_local if local else lib().ora_build_U
    f(ctypes.byref(k.s), nq or default_nq(g), _p(U))
    return U


def build_Q(g):
    k = _grid(g)
    Q = np.empty((g.nang_total, g.K))
    lib().ora_build_Q(ctypes.byref(k.s), _p(Q))
    return Q


def project(g, rho, U):
    k = _grid(g)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    B = np.empty((g.n_r, g.K))
    lib().ora_project(ctypes.byref(k.s), _p(rho), _p(np.ascontiguousarray(U)), _p(B))
    return B


def radial(g, B):
    k = _grid(g)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M = np.empty_like(B)
    lib().ora_radial(ctypes.byref(k.s), _p(B), _p(M))
    return M


def synthesize(g, M, Q):
    k = _grid(g)
    phi = np.empty(g.n_cells)
    lib().ora_synthesize(ctypes.byref(k.s), _p(np.ascontiguousarray(M)), _p(np.ascontiguousarray(Q)), _p(phi))
    return phi


def solve(g, rho, nq=None, moments=False):
    """O2: Phi on every cell; optionally also B and M."""
    k = _grid(g)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.empty(g.n_cells)
    B = np.empty((g.n_r, g.K))
    M = np.empty((g.n_r, g.K))
    rc = lib().ora_solve(ctypes.byref(k.s), nq or default_nq(g), _p(rho), _p(phi), _p(B), _p(M))
    if rc != 0:
        raise MemoryError("oracle solve failed")
    return (phi, B, M) if moments else phi


def solve_prebuilt(g, U, Q, rho):
    k = _grid(g)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.empty(g.n_cells)
    B = np.empty((g.n_r, g.K))
    M = np.empty((g.n_r, g.K))
    lib().ora_solve_prebuilt(ctypes.byref(k.s), _p(U), _p(Q), _p(rho), _p(phi), _p(B), _p(M))
    return phi


def solve_direct(g, rho, nq=None):
    """O1: brute-force addition theorem (tiny grids only)."""
    k = _grid(g)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.empty(g.n_cells)
    lib().ora_solve_direct(ctypes.byref(k.s), nq or default_nq(g), _p(rho), _p(phi))
    return phi


def solve_perpatch(g, rho, nq=None):
    """O3: the older per-patch superposition scheme."""
    k = _grid(g)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    phi = np.empty(g.n_cells)
    lib().ora_solve_perpatch(ctypes.byref(k.s), nq or default_nq(g), _p(rho), _p(phi))
    return phi


def apply_T(g, gphi, U=None, Q=None, nq=None):
    """Transpose of the linear map rho -> Phi."""
    k = _grid(g)
    U = build_U(g, nq) if U is None else U
    Q = build_Q(g) if Q is None else Q
    gphi = np.ascontiguousarray(gphi, dtype=np.float64)
    out = np.empty(g.n_cells)
    lib().ora_apply_T(ctypes.byref(k.s), _p(U), _p(Q), _p(gphi), _p(out))
    return out


def ellipsoid_phi(a, b, c, X, Y, Z, G=1.0, rho0=1.0, route="carlson"):
    f = lib().ora_ellipsoid_phi if route == "carlson" else lib().ora_ellipsoid_phi_paper
    X = np.atleast_1d(np.asarray(X, dtype=np.float64))
    Y = np.broadcast_to(np.asarray(Y, dtype=np.float64), X.shape)
    Z = np.broadcast_to(np.asarray(Z, dtype=np.float64), X.shape)
    return np.array([f(a, b, c, G, rho0, x, y, z) for x, y, z in zip(X.ravel(), Y.ravel(), Z.ravel())]).reshape(X.shape)


def carlson_rf(x, y, z):
    return lib().ora_carlson_rf(x, y, z)


def carlson_rd(x, y, z):
    return lib().ora_carlson_rd(x, y, z)
