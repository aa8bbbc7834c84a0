"""ctypes binding of libocto_fmm.so: the C ABI of include/octo_fmm.h, names unchanged.

Argument marshalling only.  The library must have been built (paper_2101_08226_gb300.build);
loading fails loudly otherwise -- there is no fallback implementation.
"""
import ctypes as C
import os

from . import build as _build

FMM_OK = 0
FMM_ERR_ARG = -1
FMM_ERR_THETA = -3
FMM_ERR_CUDA = -4
FMM_ERR_NONFINITE = -6
FMM_ERR_NOMEM = -7
FMM_ERR_STATE = -8
FMM_ERR_TIMEOUT = -9
FMM_ERR_BOUNDS = -10
FMM_FMA_F32X2 = -32  # fmm_measure_fma_rate: packed FP32 pairs
FMM_MIXED_VARIANTS = 96
FMM_NET_STATIC_MAX_POINTS = 2048 * 4096
FMM_SCF_STATE = 22
FMM_FP64 = 0
FMM_MIXED = 1
FMM_DF64 = 2

EXPORTS = [
    "fmm_build_tree", "fmm_destroy", "fmm_build_forest", "fmm_forest_info", "fmm_solve_batch", "fmm_tree_info", "fmm_tree_subgrids", "fmm_stencil",
    "fmm_interaction_counts", "fmm_interaction_counts_by_type", "fmm_last_launches", "fmm_solve", "fmm_solve_dt", "fmm_sync_status", "fmm_solve_host", "fmm_solve_host_async",
    "fmm_net_force_torque", "fmm_net_force_torque_points_static", "fmm_set_profiling", "fmm_set_graphs", "fmm_set_persistent", "fmm_set_wait_limit", "fmm_set_variant", "fmm_autotune", "fmm_binary_diagnostics", "fmm_binary_iterate", "fmm_phase_times", "fmm_measure_fma_rate", "fmm_scf_init", "fmm_scf_iterate", "fmm_partition", "fmm_ghosts", "fmm_last_error",
]

_lib = None


class ScfParams(C.Structure):
    """fmm_scf_params"""
    _fields_ = [("M1", C.c_double), ("M2", C.c_double), ("n", C.c_double), ("f", C.c_double),
                ("J0", C.c_double), ("rho_floor", C.c_double), ("theta", C.c_double),
                ("precision", C.c_int)]


class FmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"octo_fmm error {code}: {msg}")
        self.code = code


def load(path: str):
    """The library at `path` with the C ABI's signatures (the normal or the bounds-checked build)."""
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is missing: run paper_2101_08226_gb300.build.build() "
            "(there is no CPU fallback)")
    L = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "fmm_build_tree": (i32, [i32, vp, i64, C.POINTER(vp)]),
        "fmm_destroy": (None, [vp]),
        "fmm_build_forest": (i32, [vp, i32, C.POINTER(vp)]),
        "fmm_forest_info": (i32, [vp, vp, vp]),
        "fmm_solve_batch": (i32, [vp, vp, dbl, i32, i32, vp, vp, vp, vp]),
        "fmm_solve_dt": (i32, [vp, vp, vp, dbl, i32, i32, vp, vp, vp, vp, vp]),
        "fmm_tree_info": (i32, [vp, vp, vp, vp]),
        "fmm_tree_subgrids": (i32, [vp, vp]),
        "fmm_stencil": (i32, [dbl, i32, vp, i32, vp]),
        "fmm_interaction_counts": (i32, [vp, dbl, vp]),
        "fmm_interaction_counts_by_type": (i32, [vp, dbl, vp]),
        "fmm_last_launches": (i32, [vp, vp]),
        "fmm_solve": (i32, [vp, vp, dbl, i32, i32, vp, vp, vp, vp]),
        "fmm_sync_status": (i32, [vp, vp]),
        "fmm_solve_host": (i32, [vp, vp, dbl, i32, i32, vp, vp, vp, vp]),
        "fmm_solve_host_async": (i32, [vp, vp, dbl, i32, i32, vp, vp, vp, vp]),
        "fmm_net_force_torque": (i32, [vp, vp, vp, vp, vp]),
        "fmm_net_force_torque_points_static": (i32, [i64, vp, vp, vp, vp, vp]),
        "fmm_set_profiling": (i32, [vp, i32]),
        "fmm_set_graphs": (i32, [vp, i32]),
        "fmm_set_persistent": (i32, [vp, i32]),
        "fmm_set_wait_limit": (i32, [vp, C.c_longlong]),
        "fmm_set_variant": (i32, [vp, dbl, i32]),
        "fmm_autotune": (i32, [vp, vp, dbl, i32, i32, vp, vp, i32, vp, vp, vp]),
        "fmm_binary_diagnostics": (i32, [vp, vp, vp, dbl, vp, vp, dbl, dbl, vp, vp, vp]),
        "fmm_binary_iterate": (i32, [vp, vp, vp, dbl, vp, vp, i32, vp, vp, vp, vp, vp]),
        "fmm_phase_times": (i32, [vp, vp, i32]),
        "fmm_measure_fma_rate": (i32, [i32, i32, vp, vp, vp]),
        "fmm_scf_init": (i32, [vp, vp, vp, dbl, vp, vp, vp]),
        "fmm_partition": (i32, [vp, i32, i32, vp]),
        "fmm_ghosts": (i32, [vp, vp, i32, vp, i64, vp]),
        "fmm_scf_iterate": (i32, [vp, vp, i32, vp, vp, vp, vp, vp, vp]),
        "fmm_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.LIB)
    return _lib


def check(code: int) -> int:
    if code != FMM_OK:
        raise FmmError(code, lib().fmm_last_error().decode())
    return code
