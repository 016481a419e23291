"""The C ABI without a GPU: the library loads, exports every entry point
include/ygs.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import paper_1903_08475_gb300 as ygs
from paper_1903_08475_gb300 import _ygs, workloads as W
from tests._util import small_yinyang

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ygs.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(ygs_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    L = ygs.load_library()
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_ygs.EXPORTS)


def test_status_strings():
    L = ygs.load_library()
    for code, name in _ygs.STATUS.items():
        assert L.ygs_status_string(code).decode() == name


def _desc(grid, **over):
    k = dict(edges=np.ascontiguousarray(grid.edges), euler=np.ascontiguousarray(grid.euler).ravel(),
             nt=np.ascontiguousarray(grid.n_theta, np.int32), nf=np.ascontiguousarray(grid.n_phi, np.int32),
             tr=np.ascontiguousarray(grid.theta_range).ravel(), pr=np.ascontiguousarray(grid.phi_range).ravel(),
             w=np.ascontiguousarray(grid.w))
    k.update({kk: v for kk, v in over.items() if kk in k})
    dp, ip = _ygs._dp, _ygs._ip
    d = _ygs._Desc(over.get("n_r", grid.n_r), k["edges"].ctypes.data_as(dp), over.get("n_patch", grid.n_patch),
                   k["euler"].ctypes.data_as(dp), k["nt"].ctypes.data_as(ip), k["nf"].ctypes.data_as(ip),
                   k["tr"].ctypes.data_as(dp), k["pr"].ctypes.data_as(dp), k["w"].ctypes.data_as(dp),
                   over.get("l_max", grid.l_max), over.get("G", grid.G), over.get("eval", 0),
                   over.get("precision", 0), over.get("flags", 0))
    return d, k


BAD = [
    dict(n_r=0), dict(edges=np.array([0.0, 0.2, 0.1, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0, 1.1])),
    dict(edges=np.array([-0.1, 0.2, 0.3, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0, 1.1])),
    dict(n_patch=0), dict(n_patch=65), dict(nt=np.array([0, 6], np.int32)),
    dict(tr=np.array([0.5, 0.4, 0.5, 2.0])), dict(pr=np.array([0.0, 7.0, 0.0, 1.0])),
    dict(l_max=-1), dict(l_max=129), dict(G=float("nan")), dict(eval=3), dict(precision=9), dict(flags=8),
    dict(euler=np.array([0.0, float("inf"), 0, 0, 0, 0])),
]


@pytest.mark.parametrize("over", BAD)
def test_invalid_descriptor_rejected(over):
    L = ygs.load_library()
    g = small_yinyang(W)
    d, keep = _desc(g, **over)
    h = ctypes.c_void_p(1)
    st = L.ygs_create(ctypes.byref(d), 0, ctypes.byref(h))
    assert st == 1, L.ygs_last_error()
    assert h.value is None
    assert L.ygs_last_error().decode()


def test_null_arguments_rejected():
    L = ygs.load_library()
    assert L.ygs_create(None, 0, None) == 1
    assert L.ygs_solve(None, None, None, None) == 1
    assert L.ygs_backward(None, None, None, None) == 1
    assert L.ygs_solve_host_many(None, 1, None, None, None) == 1
    assert L.ygs_get_info(None, None) == 1
    assert L.ygs_destroy(None) == 0


def test_valid_descriptor_without_gpu_reports_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = ygs.load_library()
    d, keep = _desc(small_yinyang(W))
    h = ctypes.c_void_p()
    st = L.ygs_create(ctypes.byref(d), 0, ctypes.byref(h))
    assert st == 3 and h.value is None


def test_release_build_carries_no_bounds_checks():
    """The library the package loads by default is the release build; the
    checked build (index bounds checks in every per-solve kernel) lives in a
    directory of its own and is loaded only when YGS_LIB names it."""
    from paper_1903_08475_gb300 import build as B
    L = ygs.load_library()
    if os.environ.get("YGS_LIB"):
        pytest.skip("YGS_LIB selects another build")
    assert L.ygs_checked_build() == 0
    assert os.path.dirname(B.CHECKED_LIB) != os.path.dirname(B.LIB)
