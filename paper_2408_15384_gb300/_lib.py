"""ctypes declarations of libmm's C ABI (include/mm.h). Marshalling only."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmm.so")

c_i64 = ctypes.c_int64
c_u64 = ctypes.c_uint64
c_int = ctypes.c_int
c_vp = ctypes.c_void_p
c_dbl_p = ctypes.POINTER(ctypes.c_double)


class Problem(ctypes.Structure):
    _fields_ = [("m", c_i64), ("n", c_i64), ("k", c_i64),
                ("A", c_vp), ("lda", c_i64),
                ("B", c_vp), ("ldb", c_i64),
                ("C", c_vp), ("ldc", c_i64)]


class Request(ctypes.Structure):
    _fields_ = [("prob", Problem), ("precision", c_int), ("user_tag", c_u64)]


class ServeLoad(ctypes.Structure):
    _fields_ = [("count", c_i64), ("dim_lo", c_i64), ("dim_hi", c_i64), ("fp64_share", ctypes.c_double),
                ("rate_per_s", ctypes.c_double), ("seed", c_u64), ("slots", c_int), ("sample_every", c_i64)]


class ServeLoadResult(ctypes.Structure):
    _fields_ = [("completed", c_i64), ("failed", c_i64), ("wall_s", ctypes.c_double),
                ("req_per_s", ctypes.c_double), ("tflops", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p90_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("fp64_p99_ms", ctypes.c_double), ("fp32_p99_ms", ctypes.c_double)]


class ServeSample(ctypes.Structure):
    _fields_ = [("index", c_i64), ("m", c_i64), ("n", c_i64), ("k", c_i64), ("precision", c_int),
                ("slot", c_int), ("host_offset", c_i64)]


class ReqStatus(ctypes.Structure):
    _fields_ = [("status", c_int), ("user_tag", c_u64),
                ("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double),
                ("t_launch_us", ctypes.c_double), ("t_done_us", ctypes.c_double),
                ("stream", ctypes.c_int32), ("t_gpu_start_us", ctypes.c_double), ("t_gpu_end_us", ctypes.c_double)]


# name -> (restype, argtypes); the full exported surface of include/mm.h
SIGNATURES = {
    "mm_create": (c_int, [ctypes.POINTER(c_vp), c_int, ctypes.c_size_t]),
    "mm_destroy": (c_int, [c_vp]),
    "mm_status_string": (ctypes.c_char_p, [c_int]),
    "mm_gemm": (c_int, [c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_int, c_vp]),
    "mm_gemm_host": (c_int, [c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_int, c_vp]),
    "mm_sync": (c_int, [c_vp, c_vp]),
    "mm_gemm_grouped": (c_int, [c_vp, c_int, ctypes.POINTER(Problem), c_int, c_vp]),
    "mm_serve_submit": (c_int, [c_vp, ctypes.POINTER(Request), ctypes.POINTER(c_u64)]),
    "mm_serve_poll": (c_int, [c_vp, c_u64, ctypes.POINTER(ReqStatus)]),
    "mm_serve_drain": (c_int, [c_vp]),
    "mm_set_option": (c_int, [c_vp, c_int, c_i64]),
    "mm_get_option": (c_int, [c_vp, c_int, ctypes.POINTER(c_i64)]),
    "mm_slice_count_rule": (c_int, [c_i64, ctypes.c_float, ctypes.c_float]),
    "mm_crt_rule": (c_int, [c_i64, ctypes.c_float, ctypes.c_float, ctypes.POINTER(c_int)]),
    "mm_tune_save": (c_int, [c_vp, ctypes.c_char_p]),
    "mm_tune_load": (c_int, [c_vp, ctypes.c_char_p]),
    "mm_tune_lookup": (c_int, [c_vp, c_int, c_int, c_i64, c_i64, c_i64, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                               ctypes.POINTER(c_int)]),
    "mm_fill_uniform": (c_int, [c_vp, c_i64, c_i64, c_i64, c_u64, c_u64, c_int, c_u64, c_vp]),
    "mm_debug_slices": (c_int, [c_vp, c_int, c_int, c_int, c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "mm_debug_slice_count": (c_int, [c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, ctypes.POINTER(c_int),
                                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), c_vp]),
    "mm_debug_crt_residues": (c_int, [c_vp, c_int, c_int, c_int, c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "mm_gemm_emu_static_status": (c_int, [c_vp]),
    "mm_debug_crt_rebuild": (c_int, [c_vp, c_i64, c_i64, c_int, c_int, c_vp, c_vp, c_vp, c_vp, c_i64, c_vp]),
    "mm_debug_fp64_product": (c_int, [c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp,
                                      ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_float), c_vp]),
    "mm_debug_level_products": (c_int, [c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_int, c_vp, c_vp]),
    "mm_debug_level_products_int8": (c_int, [c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_int, c_vp, c_vp]),
    "mm_debug_wait_timeout": (c_int, [c_vp, c_i64, c_vp]),
    "mm_peak_fp64": (c_int, [c_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "mm_stats": (c_int, [c_vp, ctypes.POINTER(c_u64)]),
    "mm_profile_read": (c_int, [c_vp, c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_u64), c_int]),
    "mm_serve_bench": (c_int, [c_vp, ctypes.POINTER(ServeLoad), ctypes.POINTER(ServeLoadResult),
                               ctypes.POINTER(ServeSample), c_i64, ctypes.POINTER(c_i64), c_vp, c_i64]),
    "mm_gemm_emu_static": (c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_int, c_vp]),
}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmm.so; raise (never fall back) when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmm.so is not built ({path}); run `python -m paper_2408_15384_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
