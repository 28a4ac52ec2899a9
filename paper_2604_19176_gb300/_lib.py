"""ctypes declarations of the C ABI in ``include/pat.h`` (argument marshalling only).

The shared library is the in-tree ``libpatgpu.so`` built by ``build.py``.
There is no fallback: if the library is missing or fails to load, every
operator raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpatgpu.so")
DEBUG_LIB_PATH = os.path.join(_PKG, "libpatgpu_debug.so")   # -DPAT_DEBUG build (build.build(debug=True))

PAT_OK = 0
STATUS_NAMES = {
    0: "PAT_OK", 1: "PAT_ERR_INVALID_ARG", 2: "PAT_ERR_CUDA", 3: "PAT_ERR_OOM",
    4: "PAT_ERR_UNSUPPORTED", 5: "PAT_ERR_TIMEOUT", 6: "PAT_ERR_BAD_PLAN", 7: "PAT_ERR_BOUNDS",
}

# Every symbol include/pat.h declares (checked by the CPU tests).
EXPORTED = (
    "pat_plan_create", "pat_plan_destroy", "pat_plan_layout", "pat_plan_info", "pat_forward",
    "pat_adjoint", "pat_tv_grad", "pat_residual", "pat_descent_step", "pat_plan_sync_status",
    "pat_plan_set_timing", "pat_plan_kernel_times", "pat_tv_grad_noalloc", "pat_tv_step", "pat_pdhg_step",
    "pat_plan_set_wait_probe", "pat_status_string", "pat_debug_build", "pat_plan_set_bounds_probe",
    "pat_debug_fail_alloc",
)
KERNEL_KINDS = ("circmean", "abel_fwd", "abel_adj", "adjoint_gather", "tv", "residual", "descent", "tv_update",
                "pdhg_dual", "pdhg_primal", "time_pair")


class PatGeometry(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("n_det", ctypes.c_int32), ("arc_start", ctypes.c_double),
        ("arc_span", ctypes.c_double), ("n_t", ctypes.c_int32), ("t_max", ctypes.c_double),
        ("n_angles", ctypes.c_int32),
    ]


class PatOptions(ctypes.Structure):
    _fields_ = [
        ("image_dtype", ctypes.c_int32), ("schedule", ctypes.c_int32), ("tune", ctypes.c_int32),
        ("m_lanes", ctypes.c_int32), ("q_piece", ctypes.c_int32), ("band_rows", ctypes.c_int32),
        ("adj_groups", ctypes.c_int32), ("adj_mode", ctypes.c_int32), ("abel_split", ctypes.c_int32),
        ("tile_cols", ctypes.c_int32), ("time_pair", ctypes.c_int32), ("adj_jblock", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 4),
    ]


class PatPlanInfo(ctypes.Structure):
    _fields_ = [
        ("n_instances", ctypes.c_int32), ("device", ctypes.c_int32), ("f_elems", ctypes.c_int64),
        ("g_elems", ctypes.c_int64), ("samples", ctypes.c_int64), ("sample_slots", ctypes.c_int64),
        ("time_macs", ctypes.c_int64), ("work_units", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
        ("m_lanes", ctypes.c_int32), ("q_piece", ctypes.c_int32), ("band_rows", ctypes.c_int32),
        ("adj_groups", ctypes.c_int32), ("bands_max", ctypes.c_int32), ("adj_mode", ctypes.c_int32),
        ("list_bytes", ctypes.c_int64), ("abel_split_fwd", ctypes.c_int32), ("abel_split_adj", ctypes.c_int32),
        ("tile_cols", ctypes.c_int32), ("time_pair", ctypes.c_int32), ("adj_jblock", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class PatError(RuntimeError):
    def __init__(self, call: str, status: int):
        super().__init__(f"{call} failed: {STATUS_NAMES.get(status, status)}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load ``libpatgpu.so`` (or another build of it, such as the debug build at
    DEBUG_LIB_PATH) once per process and declare the prototypes; the operators
    use whichever library was loaded first (raises if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = open_library(path)
    return _lib


def open_library(path: str) -> ctypes.CDLL:
    """A separately loaded copy of a build of the library, with its prototypes."""
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the operators have no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64p = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)
    f32 = ctypes.c_float
    lib.pat_plan_create.argtypes = [ctypes.POINTER(PatGeometry), i32, ctypes.POINTER(PatOptions), vp,
                                    ctypes.POINTER(vp)]
    lib.pat_plan_destroy.argtypes = [vp]
    lib.pat_plan_layout.argtypes = [vp, i64p, i64p]
    lib.pat_plan_info.argtypes = [vp, ctypes.POINTER(PatPlanInfo)]
    lib.pat_forward.argtypes = [vp, vp, vp, vp]
    lib.pat_adjoint.argtypes = [vp, vp, vp, vp]
    lib.pat_tv_grad.argtypes = [vp, vp, f32, vp, vp, vp]
    lib.pat_residual.argtypes = [vp, vp, vp, vp, f32, vp]
    lib.pat_descent_step.argtypes = [vp, vp, vp, vp, f32, f32, i32, vp, vp]
    lib.pat_plan_sync_status.argtypes = [vp, vp]
    lib.pat_plan_set_timing.argtypes = [vp, i32]
    lib.pat_plan_set_wait_probe.argtypes = [vp, i32]
    lib.pat_plan_set_bounds_probe.argtypes = [vp, i32]
    lib.pat_debug_build.argtypes = []
    lib.pat_debug_fail_alloc.argtypes = [i32]
    lib.pat_plan_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i64p, i32]
    lib.pat_tv_grad_noalloc.argtypes = [vp, i32, i32, f32, vp, vp, vp]
    lib.pat_tv_step.argtypes = [vp, vp, vp, vp, f32, f32, f32, i32, vp, vp]
    lib.pat_pdhg_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, f32, f32, f32, i32, f32, f32, vp, vp, vp]
    lib.pat_status_string.argtypes = [i32]
    lib.pat_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name != "pat_status_string":
            getattr(lib, name).restype = ctypes.c_int
    return lib


def check(call: str, status: int) -> None:
    if status != PAT_OK:
        raise PatError(call, status)
