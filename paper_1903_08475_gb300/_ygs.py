"""ctypes binding of libygs (include/ygs.h): argument marshalling only.

Every step of a solve runs in the library's CUDA kernels; this module turns
numpy / torch objects into the plain pointers, sizes and stream handles of
the C ABI.  There is no CPU fallback: if libygs.so cannot be loaded or a call
fails, a ``YgsError`` is raised.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libygs.so")

YGS_OK = 0
STATUS = {0: "YGS_OK", 1: "YGS_ERR_INVALID_ARG", 2: "YGS_ERR_OOM", 3: "YGS_ERR_CUDA",
          4: "YGS_ERR_UNSUPPORTED", 5: "YGS_ERR_NUMERIC", 6: "YGS_ERR_TIMEOUT", 7: "YGS_ERR_BOUNDS"}
PRECISION = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "fp16x3": 3, "fp64tc": 4, "fp32": 5, "tf32x3": 6,
             "fp64emu": 7}
EVAL = {"upper_vertex": 0, "cell_centre": 1}
FLAG_NO_SYMMETRY = 1
FLAG_AUTOTUNE = 2
FLAG_CTA_PAIRS = 4

EXPORTS = ("ygs_create", "ygs_destroy", "ygs_get_info", "ygs_solve", "ygs_solve_host", "ygs_solve_host_many",
           "ygs_solve_batched",
           "ygs_backward", "ygs_get_moments", "ygs_get_weights", "ygs_get_status", "ygs_status_string",
           "ygs_last_error", "ygs_set_profiling", "ygs_read_phase_times", "ygs_launches_per_solve",
           "ygs_debug_wait_timeout", "ygs_solve_static", "ygs_batch_create", "ygs_batch_solve",
           "ygs_batch_destroy", "ygs_batch_launches", "ygs_static_scratch_capacity", "ygs_project_partial",
           "ygs_finish_from_moments", "ygs_checked_build", "ygs_debug_set_field_extent")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class YgsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("r_edges", _dp), ("n_patch", ctypes.c_int), ("euler", _dp),
                ("n_theta", _ip), ("n_phi", _ip), ("theta_range", _dp), ("phi_range", _dp),
                ("overlap_w", _dp), ("l_max", ctypes.c_int), ("G", ctypes.c_double), ("eval", ctypes.c_int),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int), ("patch_kind", _ip)]


class Info(ctypes.Structure):
    _fields_ = [("n_r", ctypes.c_int), ("n_patch", ctypes.c_int), ("l_max", ctypes.c_int), ("K", ctypes.c_int),
                ("n_ang", ctypes.c_longlong), ("n_cells", ctypes.c_longlong), ("precision", ctypes.c_int),
                ("symmetric", ctypes.c_int), ("split_k", ctypes.c_int), ("weight_bytes", ctypes.c_longlong),
                ("work_bytes", ctypes.c_longlong), ("fp64_split_k", ctypes.c_int),
                ("static_scratch_bytes", ctypes.c_longlong), ("cta_pairs", ctypes.c_int),
                ("synth_tile_shells", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load_library(path: Optional[str] = None):
    """Loads libygs.so (building it first if it is absent).  The environment
    variable YGS_LIB, when set, names another build of the library to load."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or os.environ.get("YGS_LIB") or LIB_PATH
        if not os.path.exists(p):
            from . import build as _build
            _build.build()
        L = ctypes.CDLL(p)
        vp = ctypes.c_void_p
        L.ygs_create.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.POINTER(vp)]
        L.ygs_destroy.argtypes = [vp]
        L.ygs_get_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.ygs_solve.argtypes = [vp, vp, vp, vp]
        L.ygs_solve_host.argtypes = [vp, vp, vp, vp]
        L.ygs_solve_batched.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        L.ygs_solve_host_many.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        L.ygs_backward.argtypes = [vp, vp, vp, vp]
        L.ygs_get_moments.argtypes = [vp, vp, vp, vp]
        L.ygs_get_weights.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
        L.ygs_get_status.argtypes = [vp]
        L.ygs_status_string.argtypes = [ctypes.c_int]
        L.ygs_status_string.restype = ctypes.c_char_p
        L.ygs_last_error.restype = ctypes.c_char_p
        L.ygs_set_profiling.argtypes = [vp, ctypes.c_int]
        L.ygs_read_phase_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
        L.ygs_launches_per_solve.argtypes = [vp]
        L.ygs_debug_wait_timeout.argtypes = [vp, ctypes.c_int, vp]
        L.ygs_solve_static.argtypes = [vp, vp, vp, vp]
        L.ygs_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.ygs_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
        L.ygs_batch_destroy.argtypes = [vp]
        L.ygs_batch_launches.argtypes = [vp]
        L.ygs_static_scratch_capacity.argtypes = []
        L.ygs_project_partial.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        L.ygs_finish_from_moments.argtypes = [vp, vp, vp, vp]
        L.ygs_checked_build.argtypes = []
        L.ygs_debug_set_field_extent.argtypes = [vp, ctypes.c_longlong]
        for f in EXPORTS:
            if f not in ("ygs_status_string", "ygs_last_error", "ygs_static_scratch_capacity"):
                getattr(L, f).restype = ctypes.c_int
        L.ygs_static_scratch_capacity.restype = ctypes.c_size_t
        _lib = L
        return L


def _check(st: int):
    if st != YGS_OK:
        L = load_library()
        raise YgsError(st, L.ygs_last_error().decode())


def _ptr(t) -> int:
    """Device or host address of a torch tensor / numpy array."""
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A grid plan (``ygs_create``): FP64 weights live on the device until close()."""

    def __init__(self, grid, precision: str = "fp64", device: int = 0, symmetry: bool = True,
                 autotune: bool = False, cta_pairs: bool = False):
        L = load_library()
        self._keep = keep = {
            "edges": np.ascontiguousarray(grid.edges, dtype=np.float64),
            "euler": np.ascontiguousarray(grid.euler, dtype=np.float64).reshape(-1),
            "nt": np.ascontiguousarray(grid.n_theta, dtype=np.int32),
            "nf": np.ascontiguousarray(grid.n_phi, dtype=np.int32),
            "tr": np.ascontiguousarray(grid.theta_range, dtype=np.float64).reshape(-1),
            "pr": np.ascontiguousarray(grid.phi_range, dtype=np.float64).reshape(-1),
            "w": np.ascontiguousarray(grid.w, dtype=np.float64),
        }
        kind = getattr(grid, "kind", None)
        if kind is not None:
            keep["kind"] = np.ascontiguousarray(kind, dtype=np.int32)
        d = _Desc(grid.n_r, keep["edges"].ctypes.data_as(_dp), grid.n_patch, keep["euler"].ctypes.data_as(_dp),
                  keep["nt"].ctypes.data_as(_ip), keep["nf"].ctypes.data_as(_ip), keep["tr"].ctypes.data_as(_dp),
                  keep["pr"].ctypes.data_as(_dp), keep["w"].ctypes.data_as(_dp), grid.l_max, grid.G, grid.eval,
                  PRECISION[precision], ((0 if symmetry else FLAG_NO_SYMMETRY) | (FLAG_AUTOTUNE if autotune else 0)
                   | (FLAG_CTA_PAIRS if cta_pairs else 0)),
                  keep["kind"].ctypes.data_as(_ip) if "kind" in keep else None)
        h = ctypes.c_void_p()
        _check(L.ygs_create(ctypes.byref(d), device, ctypes.byref(h)))
        self._h = h
        self.grid = grid
        self.device = device
        self.precision = precision
        inf = Info()
        _check(L.ygs_get_info(h, ctypes.byref(inf)))
        self.info = inf.as_dict()

    @property
    def handle(self):
        if self._h is None:
            raise YgsError(1, "plan is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load_library().ygs_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _field_out(plan: Plan, like):
    import torch
    return torch.empty(plan.info["n_cells"], dtype=torch.float64, device=like.device)


def ygs_solve(plan: Plan, rho, phi=None, stream=None):
    """Phi = A rho on device tensors (FP64, n_cells elements)."""
    phi = _field_out(plan, rho) if phi is None else phi
    _check(load_library().ygs_solve(plan.handle, _ptr(rho), _ptr(phi), _stream_handle(stream)))
    return phi


class Batch:
    """A fixed set of plans solved together: each group's contractions in one
    persistent launch (ygs_batch_create / ygs_batch_solve)."""

    def __init__(self, plans: Sequence[Plan]):
        L = load_library()
        n = len(plans)
        hp = (ctypes.c_void_p * n)(*[p.handle for p in plans])
        h = ctypes.c_void_p()
        _check(L.ygs_batch_create(n, hp, ctypes.byref(h)))
        self._h = h
        self.plans = list(plans)

    def solve(self, rhos, phis=None, stream=None):
        """phis[k] = A_k rhos[k] for every plan of the batch."""
        n = len(self.plans)
        if phis is None:
            phis = [_field_out(p, r) for p, r in zip(self.plans, rhos)]
        rp = (ctypes.c_void_p * n)(*[_ptr(r) for r in rhos])
        pp = (ctypes.c_void_p * n)(*[_ptr(x) for x in phis])
        _check(load_library().ygs_batch_solve(self._h, rp, pp, _stream_handle(stream)))
        return phis

    @property
    def launches(self) -> int:
        return int(load_library().ygs_batch_launches(self._h))

    def close(self):
        if self._h:
            load_library().ygs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ygs_solve_static(plan: Plan, rho, phi=None, stream=None):
    """Phi = A rho in FP64 with the library's static device scratch (no device
    allocation inside the call; the plan's info["static_scratch_bytes"] must
    be at most ygs_static_scratch_capacity())."""
    phi = _field_out(plan, rho) if phi is None else phi
    _check(load_library().ygs_solve_static(plan.handle, _ptr(rho), _ptr(phi), _stream_handle(stream)))
    return phi


def ygs_static_scratch_capacity() -> int:
    """Bytes of the device array behind ygs_solve_static (YGS_STATIC_SCRATCH_BYTES)."""
    return int(load_library().ygs_static_scratch_capacity())


def ygs_backward(plan: Plan, grad_phi, grad_rho=None, stream=None):
    """grad_rho = A^T grad_phi on device tensors."""
    grad_rho = _field_out(plan, grad_phi) if grad_rho is None else grad_rho
    _check(load_library().ygs_backward(plan.handle, _ptr(grad_phi), _ptr(grad_rho), _stream_handle(stream)))
    return grad_rho


def ygs_solve_host(plan: Plan, h_rho, h_phi, stream=None):
    """Host buffers in and out (copies inside the call); synchronous."""
    _check(load_library().ygs_solve_host(plan.handle, _ptr(h_rho), _ptr(h_phi), _stream_handle(stream)))
    return h_phi


def ygs_solve_host_many(plan: Plan, h_rhos, h_phis, stream=None):
    """n solves from and to host buffers with the copies overlapped (pinned
    CPU tensors or arrays); returns h_phis after the last result is in."""
    n = len(h_rhos)
    if len(h_phis) != n:
        raise ValueError("h_rhos and h_phis differ in length")
    VA = ctypes.c_void_p * max(n, 1)
    rp = VA(*[_ptr(r) for r in h_rhos])
    pp = VA(*[_ptr(p) for p in h_phis])
    _check(load_library().ygs_solve_host_many(plan.handle, n, rp, pp, _stream_handle(stream)))
    return h_phis


def ygs_solve_batched(plans: Sequence[Plan], rhos, phis, stream=None):
    n = len(plans)
    VA = ctypes.c_void_p * max(n, 1)
    hp = VA(*[p.handle.value for p in plans])
    rp = VA(*[_ptr(r) for r in rhos])
    pp = VA(*[_ptr(p) for p in phis])
    _check(load_library().ygs_solve_batched(n, hp, rp, pp, _stream_handle(stream)))
    return phis


def ygs_get_moments(plan: Plan, stream=None):
    import torch
    K, nr = plan.info["K"], plan.info["n_r"]
    B = torch.empty((nr, K), dtype=torch.float64, device=f"cuda:{plan.device}")
    M = torch.empty_like(B)
    _check(load_library().ygs_get_moments(plan.handle, _ptr(B), _ptr(M), _stream_handle(stream)))
    return B, M


def ygs_project_partial(plan: Plan, rho, chunk_begin: int, chunk_end: int, B=None, stream=None):
    """Moments (n_r x K, FP64, natural column order) of the cells of the plan's
    FP64 split-K chunks [chunk_begin, chunk_end) of rho: one process's share of
    an angularly sharded solve (Sect. 4.3, steps 2-3)."""
    import torch
    if B is None:
        B = torch.empty((plan.info["n_r"], plan.info["K"]), dtype=torch.float64, device=rho.device)
    _check(load_library().ygs_project_partial(plan.handle, _ptr(rho), int(chunk_begin), int(chunk_end), _ptr(B),
                                              _stream_handle(stream)))
    return B


def ygs_finish_from_moments(plan: Plan, B, out=None, stream=None):
    """Phi from the moments B of the whole field (the sum of every process's
    ygs_project_partial): radial scans and synthesis."""
    import torch
    if out is None:
        out = torch.empty(plan.info["n_cells"], dtype=torch.float64, device=B.device)
    _check(load_library().ygs_finish_from_moments(plan.handle, _ptr(B), _ptr(out), _stream_handle(stream)))
    return out


def ygs_get_weights(plan: Plan, which: str, patch: int) -> np.ndarray:
    g = plan.grid
    out = np.empty((g.nang(patch), g.K))
    _check(load_library().ygs_get_weights(plan.handle, 0 if which == "U" else 1, patch, out.ctypes.data))
    return out


def ygs_set_profiling(plan: Plan, enable: bool = True):
    _check(load_library().ygs_set_profiling(plan.handle, 1 if enable else 0))


def ygs_read_phase_times(plan: Plan):
    """Summed (field prep, projection, scans, synthesis) milliseconds and the call count."""
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int()
    _check(load_library().ygs_read_phase_times(plan.handle, ms, ctypes.byref(n)))
    return list(ms), n.value


def ygs_launches_per_solve(plan: Plan) -> int:
    return load_library().ygs_launches_per_solve(plan.handle)


def ygs_debug_wait_timeout(plan: Plan, spins: int = 1000, stream=None):
    _check(load_library().ygs_debug_wait_timeout(plan.handle, spins, _stream_handle(stream)))


def ygs_get_status(plan: Plan):
    _check(load_library().ygs_get_status(plan.handle))


def ygs_debug_set_field_extent(plan: Plan, n: int):
    """Checked builds: the field extent the kernels' bounds checks use (n_cells
    normally); a smaller one makes them report the accesses past it."""
    _check(load_library().ygs_debug_set_field_extent(plan.handle, int(n)))


def ygs_checked_build() -> bool:
    """True when the loaded library is the checked build (index bounds checks in
    every per-solve kernel, reported by ygs_get_status as YGS_ERR_BOUNDS)."""
    return bool(load_library().ygs_checked_build())


def _make_autograd():
    import torch

    class YgsSolve(torch.autograd.Function):
        """Phi = A rho with the hand-written adjoint A^T as the backward."""

        @staticmethod
        def forward(ctx, rho, plan):
            ctx.plan = plan
            return ygs_solve(plan, rho.contiguous())

        @staticmethod
        def backward(ctx, grad_phi):
            return ygs_backward(ctx.plan, grad_phi.contiguous()), None

    return YgsSolve


_autograd = None


def potential(rho, plan: Plan):
    """Differentiable Phi(rho) (torch.autograd.Function over ygs_solve / ygs_backward)."""
    global _autograd
    if _autograd is None:
        _autograd = _make_autograd()
    return _autograd.apply(rho, plan)
