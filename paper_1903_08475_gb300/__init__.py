"""GB300-native multi-patch spherical-harmonics gravity solver
(Wongwathanarat, arXiv:1903.08475).

The compute path is libygs.so (CUDA, sm_103a) behind the C ABI of
include/ygs.h; this package is its thin Python binding plus the seeded
input generators of ``workloads``.
"""
from ._ygs import (EXPORTS, LIB_PATH, Batch, Info, Plan, YgsError, load_library, potential, ygs_backward,
                   ygs_debug_wait_timeout, ygs_get_moments, ygs_get_status, ygs_get_weights, ygs_launches_per_solve,
                   ygs_read_phase_times, ygs_set_profiling, ygs_solve, ygs_solve_batched, ygs_solve_host,
                   ygs_solve_host_many, ygs_solve_static, ygs_static_scratch_capacity, ygs_project_partial,
                   ygs_finish_from_moments, ygs_checked_build, ygs_debug_set_field_extent)

__all__ = ["EXPORTS", "LIB_PATH", "Batch", "Info", "Plan", "YgsError", "load_library", "potential", "ygs_backward",
           "ygs_debug_wait_timeout", "ygs_get_moments", "ygs_get_status", "ygs_get_weights", "ygs_launches_per_solve",
           "ygs_read_phase_times", "ygs_set_profiling", "ygs_solve", "ygs_solve_batched", "ygs_solve_host",
           "ygs_solve_host_many", "ygs_solve_static", "ygs_static_scratch_capacity", "ygs_project_partial",
           "ygs_finish_from_moments", "ygs_checked_build", "ygs_debug_set_field_extent"]
