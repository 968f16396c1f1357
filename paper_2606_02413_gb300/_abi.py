"""ctypes mirror of include/rt.h and the loader of librt.so.

Argument marshalling only: every step of the ray tracing runs in the CUDA
kernels of librt.  There is no fallback: if the shared library is missing or
fails to load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librt.so")

RT_OK, RT_ERR_ARG, RT_ERR_GRID, RT_ERR_CUDA, RT_ERR_OOM, RT_ERR_TIMEOUT, RT_ERR_CHECKED, \
    RT_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
RT_F32, RT_F64 = 0, 1
RT_STEPWISE, RT_TUBE, RT_MAG_OFF = 0, 1, 2
RT_PLAIN_F32, RT_MIXED = 0, 1
RAY_STATUS = {1: "EXIT_OUTER", 2: "HIT_INNER", 3: "TAU_STOP", 4: "STEP_LIMIT", 5: "MISS", 6: "NAN"}

# every symbol include/rt.h declares
EXPORTS = ["rt_default_options", "rt_status_string", "rt_last_error", "rt_create", "rt_destroy",
           "rt_load_grid", "rt_free_grid", "rt_trace_image", "rt_backward", "rt_batch_plan_create",
           "rt_batch_plan_create_shard", "rt_shard_assign", "rt_batch_plan_launch",
           "rt_batch_plan_stats", "rt_batch_plan_destroy", "rt_trace_batch", "rt_trace_batch_noalloc",
           "rt_probe_field", "rt_disk_mean_tb", "rt_beam_convolve", "rt_trace_paths", "rt_sync", "rt_get_stats",
           "rt_trace_image_tape", "rt_backward_tape", "rt_tape_info", "rt_tape_free"]


class GridDesc(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_theta", C.c_int), ("n_phi", C.c_int),
                ("r_nodes", C.c_void_p), ("theta_nodes", C.c_void_p), ("phi_nodes", C.c_void_p),
                ("dtype", C.c_int), ("on_device", C.c_int)]


class View(C.Structure):
    _fields_ = [("lon_rad", C.c_double), ("lat_rad", C.c_double), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double)]


class Options(C.Structure):
    _fields_ = [("dtau", C.c_double), ("s_mode", C.c_int), ("n_nb", C.c_int), ("eps_mode", C.c_int),
                ("eta", C.c_double), ("delta", C.c_double), ("tau_stop", C.c_double),
                ("max_steps", C.c_int), ("tbc_mode", C.c_int), ("tbc_K", C.c_double),
                ("emission", C.c_int), ("straight", C.c_int), ("precision", C.c_int),
                ("tile", C.c_int), ("blocks_per_sm", C.c_int)]


class RayDiag(C.Structure):
    _fields_ = [("exit_pos", C.c_float * 3), ("tau", C.c_float), ("ln_s", C.c_float),
                ("steps", C.c_int32), ("status", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("view", C.POINTER(View)), ("freqs_hz", C.POINTER(C.c_double)), ("nf", C.c_int),
                ("tb_out", C.c_void_p), ("diag", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("ray_steps", C.c_ulonglong), ("rays", C.c_ulonglong)]


assert C.sizeof(RayDiag) == 28

_lock = threading.Lock()
_lib = None


def lib():
    """Load librt.so (built by ``paper_2606_02413_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librt.so is not built ({LIB_PATH}); run paper_2606_02413_gb300.build.build()")
        try:  # make the CUDA runtime that torch already loaded visible to the library
            import torch  # noqa: F401
        except Exception:
            pass
        L = C.CDLL(LIB_PATH)
        vp, ip = C.c_void_p, C.c_int
        L.rt_default_options.argtypes = [C.POINTER(Options)]
        L.rt_default_options.restype = None
        L.rt_status_string.argtypes = [ip]
        L.rt_status_string.restype = C.c_char_p
        L.rt_last_error.argtypes = []
        L.rt_last_error.restype = C.c_char_p
        L.rt_create.argtypes = [C.POINTER(vp), ip]
        L.rt_destroy.argtypes = [vp]
        L.rt_load_grid.argtypes = [vp, C.POINTER(GridDesc), vp, vp, vp, C.POINTER(vp)]
        L.rt_free_grid.argtypes = [vp, vp]
        L.rt_trace_image.argtypes = [vp, vp, C.POINTER(View), C.POINTER(C.c_double), ip,
                                     C.POINTER(Options), vp, vp, vp]
        L.rt_probe_field.argtypes = [vp, vp, vp, ip, vp, vp]
        L.rt_backward.argtypes = [vp, vp, C.POINTER(View), C.POINTER(C.c_double), ip, C.POINTER(Options),
                                  vp, vp, vp, vp, vp, vp]
        L.rt_batch_plan_create.argtypes = [vp, vp, C.POINTER(Request), ip, C.POINTER(Options), C.POINTER(vp)]
        L.rt_batch_plan_create_shard.argtypes = [vp, vp, C.POINTER(Request), ip, C.POINTER(Options), ip, ip,
                                                 C.POINTER(vp)]
        L.rt_shard_assign.argtypes = [C.POINTER(C.c_double), C.c_long, ip, C.POINTER(C.c_int)]
        L.rt_batch_plan_launch.argtypes = [vp, vp]
        L.rt_batch_plan_stats.argtypes = [vp, vp, C.POINTER(Stats)]
        L.rt_batch_plan_destroy.argtypes = [vp]
        L.rt_trace_batch.argtypes = [vp, vp, C.POINTER(Request), ip, C.POINTER(Options), vp]
        L.rt_trace_batch_noalloc.argtypes = [vp, C.POINTER(Request), ip, C.POINTER(Options), vp]
        L.rt_disk_mean_tb.argtypes = [C.POINTER(View), vp, ip, C.c_double, vp, vp]
        L.rt_beam_convolve.argtypes = [C.POINTER(View), vp, C.POINTER(C.c_double), ip, C.c_double, vp, vp, vp]
        L.rt_trace_paths.argtypes = [vp, vp, C.POINTER(View), C.c_double, C.POINTER(C.c_int), ip, C.POINTER(Options),
                                     ip, vp, vp, vp, vp, vp]
        L.rt_sync.argtypes = [vp, vp]
        L.rt_get_stats.argtypes = [vp, vp, C.POINTER(Stats)]
        L.rt_trace_image_tape.argtypes = [vp, vp, C.POINTER(View), C.POINTER(C.c_double), ip, C.POINTER(Options),
                                          C.c_size_t, vp, vp, C.POINTER(vp), vp]
        L.rt_backward_tape.argtypes = [vp, vp, vp, vp, vp]
        L.rt_tape_info.argtypes = [vp, vp, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]
        L.rt_tape_free.argtypes = [vp]
        for name in ("rt_create", "rt_destroy", "rt_load_grid", "rt_free_grid", "rt_trace_image", "rt_backward",
                     "rt_batch_plan_create", "rt_batch_plan_create_shard", "rt_shard_assign",
                     "rt_batch_plan_launch", "rt_batch_plan_stats",
                     "rt_batch_plan_destroy", "rt_trace_batch", "rt_trace_batch_noalloc", "rt_probe_field",
                     "rt_disk_mean_tb", "rt_beam_convolve", "rt_trace_paths", "rt_sync", "rt_get_stats",
                     "rt_trace_image_tape", "rt_backward_tape", "rt_tape_info", "rt_tape_free"):
            getattr(L, name).restype = ip
        _lib = L
        return _lib


class RtError(RuntimeError):
    def __init__(self, code, where):
        L = lib()
        self.code = code
        msg = L.rt_last_error().decode(errors="replace")
        super().__init__(f"{where}: {L.rt_status_string(code).decode()} ({msg})")


def check(code, where):
    if code != RT_OK:
        raise RtError(code, where)
