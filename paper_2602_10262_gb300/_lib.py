"""ctypes loader for libgb300fp8.so: argument types only, no arithmetic.

The library is built in tree by ``paper_2602_10262_gb300.build``.  There is
no fallback: if the shared object is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I64 = ctypes.c_int64
I32 = ctypes.c_int
F32 = ctypes.c_float


class FP8Problem(ctypes.Structure):
    """Mirror of ``fp8_gemm_problem`` in include/gb300fp8.h."""
    _fields_ = [
        ("M", I64), ("N", I64), ("K", I64),
        ("A", P), ("A_meta", P), ("lda", I64),
        ("B", P), ("ldb", I64),
        ("a_scale", P), ("a_mode", I32),
        ("b_scale", P), ("b_mode", I32),
        ("alpha", F32),
        ("C", P), ("ldc", I64),
        ("out_dtype", I32), ("out_transposed", I32),
        ("a_format", I32), ("b_format", I32),
    ]


class FP8QuantJob(ctypes.Structure):
    """Mirror of ``fp8_quant_job``."""
    _fields_ = [("x", P), ("rows", I64), ("cols", I64), ("ldx", I64), ("q", P), ("ldq", I64),
                ("dequant_scale", P)]


class FP8TileConfig(ctypes.Structure):
    """Mirror of ``fp8_tile_config``."""
    _fields_ = [("mt", I32), ("group_m", I32), ("ms_per_launch", F32), ("bn_max", I32)]


class FP8PlanInfo(ctypes.Structure):
    """Mirror of ``fp8_gemm_plan_info``."""
    _fields_ = [("mt", I32), ("bn", I32), ("k_blocks_per_stage", I32), ("splits", I32), ("cluster", I32),
                ("grid", I32), ("swapped", I32), ("group_m", I32), ("multicast", I32),
                ("workspace_bytes", ctypes.c_size_t)]


class FP8ServerConfig(ctypes.Structure):
    """Mirror of ``fp8_server_config``."""
    _fields_ = [("num_tenants", I32), ("latency_tenant", I32), ("batching", I32),
                ("max_batch", I32), ("max_inflight", I32), ("bulk_max_ctas", I32),
                ("pool_bytes", ctypes.c_size_t), ("reserve_bytes", ctypes.c_size_t),
                ("latency_max_batch", I32), ("latency_max_ctas", I32),
                ("latency_pool_bytes", ctypes.c_size_t)]


class FP8Request(ctypes.Structure):
    """Mirror of ``fp8_request``."""
    _fields_ = [("tenant", I32), ("weight", ctypes.c_uint64), ("M", I64), ("x", P), ("ldx", I64),
                ("out", P), ("ldo", I64), ("out_dtype", I32), ("alpha", F32)]


class FP8Result(ctypes.Structure):
    """Mirror of ``fp8_result``."""
    _fields_ = [("status", I32), ("batch_size", I32), ("t_submit_us", ctypes.c_double),
                ("t_launch_us", ctypes.c_double), ("t_end_us", ctypes.c_double),
                ("t_start_us", ctypes.c_double)]


class FP8ServerStats(ctypes.Structure):
    """Mirror of ``fp8_server_stats``."""
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("max_batch_seen", ctypes.c_uint64), ("pool_bytes", ctypes.c_size_t),
                ("pool_in_use", ctypes.c_size_t), ("pool_high_water", ctypes.c_size_t)]


SIGNATURES = {
    "fp8_status_string": (ctypes.c_char_p, [I32]),
    "fp8_last_device_error": (I32, [P]),
    "fp8_device_sm_count": (I32, []),
    "fp8_test_stall_gemm_loads": (I32, [I32, ctypes.c_double]),
    "fp8_quantize_e4m3": (I32, [P, I64, I64, I64, I32, P, I64, P, P]),
    "fp8_quantize_e5m2": (I32, [P, I64, I64, I64, I32, P, I64, P, P]),
    "fp8_mx_scale_tiled_bytes": (ctypes.c_size_t, [I64, I64]),
    "fp8_quantize_mx": (I32, [P, I64, I64, I64, I32, P, I64, P, I32, P]),
    "fp8_mx_scales_to_tiled": (I32, [P, I64, I64, P, P]),
    "gemm_fp8_mx": (I32, [I64, I64, I64, P, I64, P, P, I64, P, F32, P, I64, I32, I32, I32, P]),
    "prune24_compress": (I32, [P, I64, I64, I64, P, P, P]),
    "fp8_quantize_e4m3_prune24": (I32, [P, I64, I64, I64, P, I64, P, P, P, P]),
    "prune24_decompress": (I32, [P, P, I64, I64, P, P]),
    "gemm_fp8_dense": (I32, [I64, I64, I64, P, I64, P, I64, P, I32, P, I32, F32, P, I64, I32, P]),
    "gemm_fp8_dense_noalloc": (I32, [I64, I64, I64, P, I64, P, I64, P, I32, P, I32, F32, P, I64, I32, P]),
    "gemm_fp8_dense_fmt": (I32, [I64, I64, I64, P, I64, P, I64, P, I32, P, I32, F32, P, I64, I32,
                                 I32, I32, P]),
    "gemm_fp8_sparse24": (I32, [I64, I64, I64, P, P, P, I64, P, I32, P, I32, F32, P, I64, I32, I32, P]),
    "gemm_fp8_sparse24_fmt": (I32, [I64, I64, I64, P, P, P, I64, P, I32, P, I32, F32, P, I64, I32,
                                    I32, I32, I32, P]),
    "gemm_fp8_grouped": (I32, [ctypes.POINTER(FP8Problem), I32, P]),
    "gemm_fp8_grouped_ex": (I32, [ctypes.POINTER(FP8Problem), I32, I32, P]),
    "fp8_quantize_e4m3_rows_grouped": (I32, [ctypes.POINTER(FP8QuantJob), I32, P]),
    "fp8_gemm_set_tile_config": (I32, [I32, I32]),
    "gemm_fp8_dense_plan": (I32, [I64, I64, I64, I32, ctypes.POINTER(FP8PlanInfo)]),
    "gemm_fp8_mx_plan": (I32, [I64, I64, I64, I32, ctypes.POINTER(FP8PlanInfo)]),
    "gemm_fp8_sparse24_plan": (I32, [I64, I64, I64, I32, ctypes.POINTER(FP8PlanInfo)]),
    "fp8_gemm_set_multicast": (I32, [I32]),
    "gemm_fp8_grouped_autotune": (I32, [ctypes.POINTER(FP8Problem), I32, I32, I32, P,
                                        ctypes.POINTER(FP8TileConfig)]),
    "gemm_fp8_tune_cache_save": (I32, [ctypes.c_char_p]),
    "gemm_fp8_tune_cache_load": (I32, [ctypes.c_char_p]),
    "gemm_fp8_tune_cache_clear": (I32, []),
    "gemm_fp8_grouped_graph_create": (I32, [ctypes.POINTER(FP8Problem), I32, I32, ctypes.POINTER(P)]),
    "gemm_fp8_grouped_graph_update": (I32, [P, ctypes.POINTER(FP8Problem), I32]),
    "gemm_fp8_grouped_graph_launch": (I32, [P, P]),
    "gemm_fp8_grouped_graph_destroy": (I32, [P]),
    "fp8_server_create": (I32, [ctypes.POINTER(FP8ServerConfig), ctypes.POINTER(P)]),
    "fp8_server_create_simulated": (I32, [ctypes.POINTER(FP8ServerConfig), ctypes.c_double,
                                          ctypes.c_double, I32, ctypes.POINTER(P)]),
    "fp8_server_destroy": (I32, [P]),
    "fp8_server_register_weight": (I32, [P, I64, I64, P, I64, P, P, I32,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "fp8_server_register_weight_fmt": (I32, [P, I64, I64, P, I64, P, P, I32, I32,
                                             ctypes.POINTER(ctypes.c_uint64)]),
    "fp8_server_submit": (I32, [P, ctypes.POINTER(FP8Request), ctypes.POINTER(ctypes.c_uint64)]),
    "fp8_server_poll": (I32, [P, ctypes.c_uint64, ctypes.POINTER(FP8Result)]),
    "fp8_server_wait": (I32, [P, ctypes.c_uint64, ctypes.POINTER(FP8Result), ctypes.c_double]),
    "fp8_server_get_stats": (I32, [P, ctypes.POINTER(FP8ServerStats)]),
    "fp8_server_now_us": (ctypes.c_double, [P]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) and return the CDLL."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgb300fp8.so not found at {path}; run the build first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib
