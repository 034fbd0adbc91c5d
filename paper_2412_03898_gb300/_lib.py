"""ctypes declarations of the C ABI in include/pa.h (libpa.so, built in-tree).

Argument marshalling only.  Importing this module loads the CUDA library and
raises if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpa.so")

PA_OK = 0
PA_ERR_INVALID_ARG = 1
PA_ERR_DOMAIN = 2
PA_ERR_CUDA = 3
PA_ERR_TIMEOUT = 4
PA_ERR_WORKSPACE = 5
PA_ACCUMULATE = 1
PA_SSIM_MINMAX = 4
PA_PROFILE_UNIFORM = 2
PA_PLAN_TUNE = 8
PA_ADJOINT_WORKSPACE_BYTES = 256

c_float_p = ctypes.c_void_p  # device pointers travel as void*


class pa_geom(ctypes.Structure):
    _fields_ = [("sensors", ctypes.c_void_p), ("n_sensors", ctypes.c_int32), ("sensor_stride", ctypes.c_int32),
                ("c", ctypes.c_float), ("fs", ctypes.c_float), ("t0", ctypes.c_float),
                ("n_samples", ctypes.c_int32), ("kappa", ctypes.c_float)]


class pa_balls(ctypes.Structure):
    _fields_ = [("state", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int64)]


class pa_canon(ctypes.Structure):
    _fields_ = [("canon", ctypes.c_void_p), ("omega", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("n", ctypes.c_int64), ("stride", ctypes.c_int64),
                ("n_basis", ctypes.c_int32)]


class pa_grads(ctypes.Structure):
    _fields_ = [("state", ctypes.c_void_p), ("omega", ctypes.c_void_p), ("theta", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p)]


class pa_scene(ctypes.Structure):
    _fields_ = [("geom", pa_geom), ("balls", pa_balls), ("n_frames", ctypes.c_int32), ("traces", ctypes.c_void_p),
                ("trace_grad", ctypes.c_void_p), ("grad_state", ctypes.c_void_p)]


PA_MAX_SCENES = 64


class pa_grid(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("h", ctypes.c_float), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32)]


class PAError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


_lib = None


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpa.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python paper_2412_03898_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i32, i64, u32, f32, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float, ctypes.c_size_t
    G, B, C, GR = (ctypes.POINTER(pa_geom), ctypes.POINTER(pa_balls), ctypes.POINTER(pa_canon),
                   ctypes.POINTER(pa_grads))
    I32P = ctypes.POINTER(ctypes.c_int32)
    sig = {
        "pa_status_string": (ctypes.c_char_p, [i32]),
        "pa_version": (i32, []),
        "pa_device_error": (i32, [P, I32P]),
        "pa_deform_balls": (i32, [C, P, i32, P, P]),
        "pa_deform_backward": (i32, [C, P, i32, P, GR, u32, P]),
        "pa_forward_workspace_size": (sz, [G, B, i32]),
        "pa_forward_workspace_size_ex": (sz, [G, B, i32, I32P]),
        "pa_forward": (i32, [G, B, i32, P, u32, P, sz, P]),
        "pa_forward_ex": (i32, [G, B, i32, P, u32, I32P, P, sz, P]),
        "pa_forward_plan_info": (i32, [G, B, i32, I32P, I32P]),
        "pa_adjoint": (i32, [G, B, C, P, i32, P, P, GR, u32, P, sz, P]),
        "pa_batched_workspace_size": (sz, [ctypes.POINTER(pa_scene), i32, P]),
        "pa_forward_batched": (i32, [ctypes.POINTER(pa_scene), i32, u32, P, P, sz, P]),
        "pa_adjoint_batched": (i32, [ctypes.POINTER(pa_scene), i32, u32, P, P, sz, P]),
        "pa_plan_workspace_size": (sz, [ctypes.POINTER(pa_scene), i32]),
        "pa_plan_create": (i32, [ctypes.POINTER(pa_scene), i32, u32, P, sz, P, ctypes.POINTER(P)]),
        "pa_plan_from_values": (i32, [I32P, ctypes.POINTER(P)]),
        "pa_plan_get": (i32, [P, I32P, ctypes.POINTER(ctypes.c_float)]),
        "pa_plan_destroy": (None, [P]),
        "pa_forward_4d_workspace_size": (sz, [G, C, i32, P]),
        "pa_forward_4d": (i32, [G, C, P, i32, P, u32, P, P, sz, P]),
        "pa_adjoint_4d_workspace_size": (sz, [G, C, i32, P]),
        "pa_adjoint_4d": (i32, [G, C, P, i32, P, P, GR, u32, P, P, sz, P]),
        "pa_spatial_order_workspace_size": (sz, [i64]),
        "pa_spatial_order": (i32, [B, P, P, sz, P]),
        "pa_gather_rows": (i32, [P, P, i64, i64, i32, P, P]),
        "pa_loss_workspace_size": (sz, [i64, i32]),
        "pa_residual_loss": (i32, [P, P, i64, i32, P, P, P, P, sz, P]),
        "pa_residual_loss_noalloc": (i32, [P, P, i64, i32, P, P, P, P]),
        "pa_sumsq": (i32, [P, i64, P, P, sz, P]),
        "pa_count_contributions": (i32, [G, B, i32, P, P]),
        "pa_adam_step": (i32, [P, P, P, P, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32, P]),
        "pa_adam_step_scheduled": (i32, [P, P, P, P, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, i32, ctypes.c_double, P, P]),
        "pa_step_increment": (i32, [P, P]),
        "pa_ubp_filter": (i32, [P, i64, i32, f32, f32, P, P]),
        "pa_ubp": (i32, [G, ctypes.POINTER(ctypes.c_float), P, ctypes.POINTER(pa_grid), P, P]),
        "pa_splat": (i32, [B, f32, ctypes.POINTER(pa_grid), P, P]),
        "pa_map": (i32, [P, ctypes.POINTER(pa_grid), P, P, P, P]),
        "pa_ssim_workspace_size": (sz, [i32, i32]),
        "pa_ssim": (i32, [P, P, i32, i32, f32, u32, P, P, P, sz, P]),
        "pa_selftest_bounded_wait": (i32, [ctypes.c_uint64, P]),
        "pa_measure_unit_rates": (i32, [P, ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().pa_status_string(int(status)).decode()
    except Exception:  # pragma: no cover
        return f"status {status}"


def check(status: int, where: str) -> None:
    if status != PA_OK:
        raise PAError(status, where)


def exported_symbols() -> list[str]:
    """Names of the C-ABI entry points declared in this module."""
    return ["pa_status_string", "pa_version", "pa_device_error", "pa_deform_balls", "pa_deform_backward",
            "pa_forward_workspace_size",
            "pa_forward_workspace_size_ex", "pa_forward", "pa_forward_ex", "pa_forward_plan_info", "pa_adjoint",
            "pa_batched_workspace_size", "pa_forward_batched", "pa_adjoint_batched", "pa_plan_workspace_size",
            "pa_plan_create", "pa_plan_from_values", "pa_plan_get", "pa_plan_destroy",
            "pa_forward_4d_workspace_size", "pa_forward_4d", "pa_adjoint_4d_workspace_size", "pa_adjoint_4d",
            "pa_spatial_order_workspace_size", "pa_spatial_order", "pa_gather_rows",
            "pa_loss_workspace_size", "pa_residual_loss", "pa_residual_loss_noalloc", "pa_sumsq", "pa_count_contributions", "pa_adam_step",
            "pa_adam_step_scheduled", "pa_step_increment", "pa_ubp_filter", "pa_ubp", "pa_splat", "pa_map",
            "pa_ssim_workspace_size", "pa_ssim", "pa_selftest_bounded_wait", "pa_measure_unit_rates"]
