"""ctypes declarations of the C ABI in include/scw.h and include/scw_fno.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_size_t, c_uint, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libscw.so")

SCW_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARGUMENT", 2: "UNSUPPORTED", 3: "OUT_OF_MEMORY", 4: "CUDA",
                5: "TIMEOUT", 6: "NUMERIC", 7: "STATE", 8: "BOUNDS"}
PRECISION = {"fp32": 0, "split_bf16": 1, "fp16": 2}
FLAG_EXTERIOR = 1
FLAG_HOST_IO = 2
FLAG_AUTOTUNE = 4
FLAG_DEBUG_BOUNDS = 8


class ScwDesc(ctypes.Structure):
    _fields_ = [("U", c_int), ("V", c_int), ("L", c_int),
                ("lam", c_double), ("X", c_double), ("Y", c_double),
                ("z_bounds", POINTER(c_double)),
                ("Fx", c_int), ("Fy", c_int), ("Fz", c_int),
                ("z_planes", POINTER(c_double)),
                ("x0", c_double), ("y0", c_double),
                ("n_top", c_double), ("n_bot_re", c_double), ("n_bot_im", c_double),
                ("z_inc", c_double),
                ("precision", c_int), ("flags", c_uint), ("k_split", c_int),
                ("illuminations", c_int), ("pupil_na", c_double),
                ("tiles_x", c_int), ("tiles_y", c_int),
                ("out_ld", ctypes.c_longlong), ("out_plane_stride", ctypes.c_longlong)]


class ScwPlanInfo(ctypes.Structure):
    _fields_ = [("M", c_int), ("active_layers", c_int), ("planes_per_layer_pad", c_int),
                ("k_split", c_int), ("exterior_planes", c_int), ("workspace_bytes", c_size_t),
                ("convert_ms", c_double), ("kernels_per_synthesis", c_int), ("items", c_int),
                ("contract_ctas", c_int), ("contract_tasks", c_int), ("schedule_max_load", c_double),
                ("schedule_mean_load", c_double)]


class ScwFnoDesc(ctypes.Structure):
    _fields_ = [("width", c_int), ("grid", c_int), ("modes", c_int), ("layers", c_int), ("slices", c_int),
                ("in_grid", c_int), ("batch_max", c_int), ("precision", c_int), ("seed", ctypes.c_ulonglong)]


FNO_PRECISION = {"bf16": 0, "fp32": 1}


class ScwFnoTimes(ctypes.Structure):
    _fields_ = [("calls", c_int), ("dft_ms", c_double), ("layer_ms", c_double), ("dw_ms", c_double),
                ("mix_ms", c_double), ("other_ms", c_double), ("total_ms", c_double), ("dft_flops", c_double),
                ("layer_flops", c_double), ("dw_flops", c_double), ("mix_flops", c_double)]


class ScwKernelTimes(ctypes.Structure):
    _fields_ = [("calls", c_int), ("phases_ms", c_double), ("contract_ms", c_double), ("recompose_ms", c_double),
                ("xpass_ms", c_double), ("ypass_ms", c_double), ("total_ms", c_double)]


class ScwSolveDesc(ctypes.Structure):
    _fields_ = [("U", c_int), ("V", c_int), ("L", c_int), ("lam", c_double), ("X", c_double), ("Y", c_double),
                ("z_bounds", POINTER(c_double)), ("Nx", c_int), ("Ny", c_int), ("n_top", c_double),
                ("n_bot_re", c_double), ("n_bot_im", c_double), ("z_inc", c_double)]


class ScwSolveTimes(ctypes.Structure):
    _fields_ = [("calls", c_int), ("fourier_ms", c_double), ("modes_ms", c_double), ("connect_ms", c_double),
                ("system_ms", c_double), ("alpha_ms", c_double), ("erows_ms", c_double), ("total_ms", c_double)]


# name -> (restype, argtypes); mirrors include/scw.h, include/scw_fno.h and include/scw_solve.h
SIGNATURES = {
    "scw_plan_create": (c_int, [POINTER(ScwDesc), POINTER(c_void_p)]),
    "scw_plan": (c_int, [POINTER(ScwDesc), c_void_p, POINTER(c_void_p)]),
    "scw_plan_enable_trace": (c_int, [c_void_p, c_int]),
    "scw_plan_debug_set_extent": (c_int, [c_void_p, c_int, ctypes.c_ulonglong]),
    "scw_plan_get_trace": (c_int, [c_void_p, POINTER(ctypes.c_double), c_int]),
    "scw_plan_destroy": (c_int, [c_void_p]),
    "scw_plan_set_layers": (c_int, [c_void_p] + [c_void_p] * 6 + [c_void_p]),
    "scw_synthesize": (c_int, [c_void_p, c_void_p, c_void_p]),
    "scw_spectrum": (c_int, [c_void_p, c_void_p, c_void_p]),
    "scw_recompose": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "scw_plan_set_points": (c_int, [c_void_p, c_void_p, c_int]),
    "scw_synthesize_points": (c_int, [c_void_p, c_void_p, c_void_p]),
    "scw_plan_set_point_planes": (c_int, [c_void_p, c_void_p]),
    "scw_synthesize_host": (c_int, [c_void_p] + [c_void_p] * 7 + [c_void_p]),
    "scw_plan_batched_create": (c_int, [POINTER(ScwDesc), c_int, POINTER(c_void_p)]),
    "scw_plan_batched": (c_int, [POINTER(ScwDesc), c_int, c_void_p, POINTER(c_void_p)]),
    "scw_plan_batched_set_layers": (c_int, [c_void_p, c_int] + [c_void_p] * 6 + [c_void_p]),
    "scw_synthesize_batched": (c_int, [c_void_p, c_void_p, POINTER(c_void_p), c_void_p]),
    "scw_plan_tune_report": (c_char_p, [c_void_p]),
    "scw_plan_set_pipeline": (c_int, [c_void_p, c_int]),
    "scw_plan_check": (c_int, [c_void_p, c_void_p]),
    "scw_plan_set_timeout_ns": (c_int, [c_void_p, c_uint64]),
    "scw_plan_inject_stall": (c_int, [c_void_p, c_int]),
    "scw_plan_get_info": (c_int, [c_void_p, POINTER(ScwPlanInfo)]),
    "scw_plan_enable_timing": (c_int, [c_void_p, c_int]),
    "scw_plan_get_timings": (c_int, [c_void_p, POINTER(ScwKernelTimes)]),
    "scw_recompose_noalloc": (c_int, [c_int, c_int, c_double, c_double, c_int, c_int, c_int, c_double, c_double,
                                      c_void_p, c_void_p, c_void_p]),
    "scw_surrogate_create": (c_int, [POINTER(ScwFnoDesc), POINTER(c_void_p)]),
    "scw_surrogate_destroy": (c_int, [c_void_p]),
    "scw_surrogate_param_count": (c_int, [c_void_p, POINTER(c_size_t)]),
    "scw_surrogate_set_params": (c_int, [c_void_p, c_void_p, c_size_t]),
    "scw_surrogate_get_params": (c_int, [c_void_p, c_void_p, c_size_t]),
    "scw_surrogate_get_grads": (c_int, [c_void_p, c_void_p, c_size_t]),
    "scw_surrogate_forward_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "scw_surrogate_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, c_void_p, c_void_p]),
    "scw_surrogate_infer": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, ctypes.c_float,
                                    c_void_p]),
    "scw_surrogate_calibrate": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, c_void_p]),
    "scw_surrogate_set_offset": (c_int, [c_void_p, ctypes.c_float]),
    "scw_surrogate_launches": (c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    "scw_surrogate_enable_timing": (c_int, [c_void_p, c_int]),
    "scw_surrogate_state_bytes": (c_int, [c_void_p, POINTER(c_size_t)]),
    "scw_surrogate_save_state": (c_int, [c_void_p, c_void_p, c_size_t]),
    "scw_surrogate_load_state": (c_int, [c_void_p, c_void_p, c_size_t]),
    "scw_surrogate_get_timings": (c_int, [c_void_p, POINTER(ScwFnoTimes)]),
    "scw_solver_create": (c_int, [POINTER(ScwSolveDesc), POINTER(c_void_p)]),
    "scw_solver_destroy": (c_int, [c_void_p]),
    "scw_solver_incident": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "scw_solve": (c_int, [c_void_p] + [c_void_p] * 7 + [c_void_p]),
    "scw_solver_get_times": (c_int, [c_void_p, POINTER(ScwSolveTimes)]),
    "scw_status_string": (c_char_p, [c_int]),
    "scw_last_error": (c_char_p, []),
    "scw_version": (c_int, []),
}

_lib = None


class ScwError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def load():
    """Load libscw.so from the package directory; raises if it was never built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2404_07293_gb300.build` "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int, where: str) -> None:
    if status != SCW_OK:
        msg = load().scw_last_error()
        raise ScwError(status, where, msg.decode() if msg else "")
