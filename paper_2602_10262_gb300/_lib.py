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
    ]


SIGNATURES = {
    "fp8_status_string": (ctypes.c_char_p, [I32]),
    "fp8_last_device_error": (I32, [P]),
    "fp8_device_sm_count": (I32, []),
    "fp8_quantize_e4m3": (I32, [P, I64, I64, I64, I32, P, I64, P, P]),
    "prune24_compress": (I32, [P, I64, I64, I64, P, P, P]),
    "prune24_decompress": (I32, [P, P, I64, I64, P, P]),
    "gemm_fp8_dense": (I32, [I64, I64, I64, P, I64, P, I64, P, I32, P, I32, F32, P, I64, I32, P]),
    "gemm_fp8_sparse24": (I32, [I64, I64, I64, P, P, P, I64, P, I32, P, I32, F32, P, I64, I32, I32, P]),
    "gemm_fp8_grouped": (I32, [ctypes.POINTER(FP8Problem), I32, P]),
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
