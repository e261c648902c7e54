"""CPU oracle for the FP8 (E4M3 / E5M2) dense / 2:4-sparse GEMM path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the product library never imports, links or runs it.
It shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C, FP64 accumulation, OpenMP over
output rows); this module compiles it with gcc on first use and wraps it with
numpy arrays.  Each wrapper names the definition it follows (arXiv 2602.10262:
section 2 "FP8 Matrix Cores" for the E4M3 and E5M2 formats and FP8 x FP8 ->
wide accumulation, Table 3 for mixed-format operand pairs, section 2
"Structured Sparsity" and section 6 for 2:4 sparsity; block-scaled FP8
with E8M0 scales per 32 elements follows the OCP MX layout and is not in
the paper).  Format numbers: ``E4M3 = 0``, ``E5M2 = 1``.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (exhaustive decode, brute-force encode, closed-form
quantisation fixtures, hand-built 2:4 groups, numpy float64 matmul on decoded
inputs, identity and permutation invariants, the defining property of the
block scales); ``tests/test_oracle_mutants.py``
shows that planted mistakes in ``oracle.c`` fail those pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


class OracleError(ValueError):
    pass


def compile_library(src: str, out: str) -> str:
    """gcc, OpenMP, no FP contraction (every fp32 multiply and divide is a
    single IEEE operation)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it if stale."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(SOURCE)):
        return _LIB
    return compile_library(SOURCE, _LIB)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype):
    return np.require(np.asarray(a, dtype=dtype), requirements="C")


def _scales(s, n, mode):
    s = _c(np.atleast_1d(s), np.float32)
    if s.size < (n if mode else 1):
        raise OracleError("scale vector too short")
    return s


class Oracle:
    """numpy front end over one compiled copy of ``oracle.c``."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.orc_e4m3_decode.restype = ctypes.c_double
        lib.orc_e4m3_decode.argtypes = [ctypes.c_uint8]
        lib.orc_e5m2_decode.restype = ctypes.c_double
        lib.orc_e5m2_decode.argtypes = [ctypes.c_uint8]
        for name in ("orc_e4m3_encode", "orc_e4m3_encode_bruteforce", "orc_e4m3_encode_search",
                     "orc_e5m2_encode", "orc_e5m2_encode_bruteforce", "orc_e5m2_encode_search"):
            getattr(lib, name).restype = ctypes.c_uint8
            getattr(lib, name).argtypes = [ctypes.c_float]
        for f in ("e4m3", "e5m2"):
            getattr(lib, f"orc_{f}_decode_array").argtypes = [P, i64, P]
            getattr(lib, f"orc_{f}_encode_array").argtypes = [P, i64, P]
        for name in ("orc_check_encoder_range", "orc_check_e5m2_encoder_range"):
            getattr(lib, name).restype = i64
            getattr(lib, name).argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.POINTER(ctypes.c_uint32)]
        for name in ("orc_encode_pattern_range", "orc_e5m2_encode_pattern_range"):
            getattr(lib, name).argtypes = [ctypes.c_uint64, ctypes.c_uint64, P]
        lib.orc_quantize_fmt.restype = i32
        lib.orc_quantize_fmt.argtypes = [P, i64, i64, i64, i32, i32, P, i64, P]
        lib.orc_prune24.restype = i32
        lib.orc_prune24.argtypes = [P, i64, i64, i64, P, P]
        lib.orc_decompress24.argtypes = [P, P, i64, i64, P]
        lib.orc_gemm.argtypes = [i64, i64, i64, P, i64, P, i64, P, i32, P, i32,
                                 ctypes.c_double, i32, i32, P]
        lib.orc_gemm_sampled.argtypes = [i64, P, i64, P, i64, P, i32, P, i32,
                                         ctypes.c_double, i32, i32, i64, P, P, P]
        lib.orc_gemm_sparse24.argtypes = [i64, i64, i64, P, P, P, i64, P, i32, P, i32,
                                          ctypes.c_double, i32, i32, P]
        lib.orc_e8m0_decode_array.argtypes = [P, i64, P]
        lib.orc_mx_quantize.restype = i32
        lib.orc_mx_quantize.argtypes = [P, i64, i64, i64, i32, P, i64, P]
        lib.orc_gemm_mx.argtypes = [i64, i64, i64, P, i64, P, P, i64, P, ctypes.c_double, i32, i32,
                                    P]
        lib.orc_max_threads.restype = i32
        lib.orc_set_threads.argtypes = [i32]
        self.lib = lib

    # --- E4M3 codec (OCP E4M3; paper section 2) ------------------------------

    def e4m3_decode(self, codes) -> np.ndarray:
        """Decode E4M3 codes to float64 by the OCP bit layout."""
        c = _c(codes, np.uint8)
        out = np.empty(c.shape, np.float64)
        self.lib.orc_e4m3_decode_array(_ptr(c), c.size, _ptr(out))
        return out

    def e4m3_encode(self, x) -> np.ndarray:
        """fp32 -> E4M3 code, round to nearest even, saturating to +-448."""
        a = _c(x, np.float32)
        out = np.empty(a.shape, np.uint8)
        self.lib.orc_e4m3_encode_array(_ptr(a), a.size, _ptr(out))
        return out

    def e4m3_encode_bruteforce(self, x: float) -> int:
        """Nearest finite code by a linear scan over every code (ties: even)."""
        return int(self.lib.orc_e4m3_encode_bruteforce(ctypes.c_float(x)))

    def e4m3_encode_search(self, x: float) -> int:
        """Nearest finite code located by bisection (same definition)."""
        return int(self.lib.orc_e4m3_encode_search(ctypes.c_float(x)))

    def check_encoder_range(self, lo: int, hi: int):
        """Arithmetic encoder vs nearest-value search over fp32 bit patterns
        [lo, hi).  Returns (mismatches, first bad pattern or 0xFFFFFFFF)."""
        first = ctypes.c_uint32(0)
        bad = self.lib.orc_check_encoder_range(lo, hi, ctypes.byref(first))
        return int(bad), int(first.value)

    def encode_pattern_range(self, lo: int, hi: int) -> np.ndarray:
        """Codes of every fp32 bit pattern in [lo, hi)."""
        out = np.empty(hi - lo, np.uint8)
        self.lib.orc_encode_pattern_range(lo, hi, _ptr(out))
        return out

    # --- E5M2 codec (OCP E5M2; paper section 2 "bf8") --------------------------

    def e5m2_decode(self, codes) -> np.ndarray:
        """Decode E5M2 codes to float64 by the OCP bit layout (inf and NaN
        codes decode to inf and NaN)."""
        c = _c(codes, np.uint8)
        out = np.empty(c.shape, np.float64)
        self.lib.orc_e5m2_decode_array(_ptr(c), c.size, _ptr(out))
        return out

    def e5m2_encode(self, x) -> np.ndarray:
        """fp32 -> E5M2 code, round to nearest even, saturating to +-57344."""
        a = _c(x, np.float32)
        out = np.empty(a.shape, np.uint8)
        self.lib.orc_e5m2_encode_array(_ptr(a), a.size, _ptr(out))
        return out

    def e5m2_encode_bruteforce(self, x: float) -> int:
        return int(self.lib.orc_e5m2_encode_bruteforce(ctypes.c_float(x)))

    def e5m2_encode_search(self, x: float) -> int:
        return int(self.lib.orc_e5m2_encode_search(ctypes.c_float(x)))

    def check_e5m2_encoder_range(self, lo: int, hi: int):
        first = ctypes.c_uint32(0)
        bad = self.lib.orc_check_e5m2_encoder_range(lo, hi, ctypes.byref(first))
        return int(bad), int(first.value)

    def e5m2_encode_pattern_range(self, lo: int, hi: int) -> np.ndarray:
        out = np.empty(hi - lo, np.uint8)
        self.lib.orc_e5m2_encode_pattern_range(lo, hi, _ptr(out))
        return out

    def decode(self, codes, fmt: int) -> np.ndarray:
        """Decode codes of format fmt (0: E4M3, 1: E5M2)."""
        return self.e5m2_decode(codes) if fmt == 1 else self.e4m3_decode(codes)

    # --- quantisation ---------------------------------------------------------

    def quantize(self, x, mode: int, fmt: int = 0):
        """Scale selection + encode.  mode 0 = per tensor, 1 = per row; fmt 0 =
        E4M3 (amax -> 448), 1 = E5M2 (amax -> 57344).
        Returns (codes uint8 [R, C], dequant scales float32 [1] or [R])."""
        a = _c(x, np.float32)
        if a.ndim != 2:
            raise OracleError("quantize expects a 2-D array")
        R, C = a.shape
        q = np.empty((R, C), np.uint8)
        d = np.empty(1 if mode == 0 else R, np.float32)
        if fmt not in (0, 1):
            raise OracleError("fmt must be 0 (E4M3) or 1 (E5M2)")
        rc = self.lib.orc_quantize_fmt(_ptr(a), R, C, C, int(mode), int(fmt), _ptr(q), C,
                                       _ptr(d))
        if rc == -4:
            raise OracleError("non-finite input")
        return q, d

    # --- 2:4 prune / compress ---------------------------------------------------

    def prune24(self, a):
        """Keep the two largest magnitudes of each group of four along K.
        Returns (vals uint8 [M, K/2], meta uint8 [M, ceil(K/8)])."""
        c = _c(a, np.uint8)
        M, K = c.shape
        if K % 4:
            raise OracleError("K must be a multiple of 4")
        vals = np.empty((M, K // 2), np.uint8)
        meta = np.empty((M, (K + 7) // 8), np.uint8)
        self.lib.orc_prune24(_ptr(c), M, K, K, _ptr(vals), _ptr(meta))
        return vals, meta

    def decompress24(self, vals, meta, K: int) -> np.ndarray:
        v = _c(vals, np.uint8)
        m = _c(meta, np.uint8)
        out = np.empty((v.shape[0], K), np.uint8)
        self.lib.orc_decompress24(_ptr(v), _ptr(m), v.shape[0], K, _ptr(out))
        return out

    # --- GEMM ---------------------------------------------------------------

    def gemm(self, A, B, dA, a_mode, dB, b_mode, alpha=1.0, a_fmt=0, b_fmt=0) -> np.ndarray:
        """C = alpha * dA[m] * dB[n] * sum_k decA(A[m,k]) decB(B[n,k]) in FP64.
        A: codes [M, K] of format a_fmt; B: codes [N, K] of format b_fmt."""
        A = _c(A, np.uint8)
        B = _c(B, np.uint8)
        M, K = A.shape
        N, K2 = B.shape
        if K != K2:
            raise OracleError("K mismatch")
        sa, sb = _scales(dA, M, a_mode), _scales(dB, N, b_mode)
        C = np.empty((M, N), np.float64)
        self.lib.orc_gemm(M, N, K, _ptr(A), K, _ptr(B), K, _ptr(sa), int(a_mode),
                          _ptr(sb), int(b_mode), float(alpha), int(a_fmt), int(b_fmt), _ptr(C))
        return C

    def gemm_sampled(self, A, B, dA, a_mode, dB, b_mode, alpha, ms, ns, a_fmt=0,
                     b_fmt=0) -> np.ndarray:
        """The GEMM definition at the (ms[i], ns[i]) entries only."""
        A = _c(A, np.uint8)
        B = _c(B, np.uint8)
        M, K = A.shape
        N = B.shape[0]
        ms = _c(ms, np.int64)
        ns = _c(ns, np.int64)
        if ms.size and (ms.min() < 0 or ms.max() >= M or ns.min() < 0 or ns.max() >= N):
            raise OracleError("sample index out of range")
        sa, sb = _scales(dA, M, a_mode), _scales(dB, N, b_mode)
        out = np.empty(ms.size, np.float64)
        self.lib.orc_gemm_sampled(K, _ptr(A), K, _ptr(B), K, _ptr(sa), int(a_mode),
                                  _ptr(sb), int(b_mode), float(alpha), int(a_fmt), int(b_fmt),
                                  ms.size,
                                  _ptr(ms), _ptr(ns), _ptr(out))
        return out

    def gemm_sparse24(self, vals, meta, B, K, dA, a_mode, dB, b_mode, alpha=1.0, a_fmt=0,
                      b_fmt=0):
        """Sparse GEMM = dense GEMM of the decompressed pruned A."""
        v = _c(vals, np.uint8)
        m = _c(meta, np.uint8)
        B = _c(B, np.uint8)
        M, N = v.shape[0], B.shape[0]
        sa, sb = _scales(dA, M, a_mode), _scales(dB, N, b_mode)
        C = np.empty((M, N), np.float64)
        self.lib.orc_gemm_sparse24(M, N, K, _ptr(v), _ptr(m), _ptr(B), K, _ptr(sa),
                                   int(a_mode), _ptr(sb), int(b_mode), float(alpha), int(a_fmt),
                                   int(b_fmt), _ptr(C))
        return C

    # --- block-scaled FP8 (OCP MX; not in the paper) --------------------------

    def e8m0_decode(self, codes) -> np.ndarray:
        """E8M0 scale codes -> 2^(code - 127) (0xFF: NaN)."""
        c = _c(codes, np.uint8)
        out = np.empty(c.shape, np.float64)
        self.lib.orc_e8m0_decode_array(_ptr(c), c.size, _ptr(out))
        return out

    def mx_quantize(self, x, fmt: int = 0):
        """fp32 [R, C] (C % 32 == 0) -> (codes uint8 [R, C], E8M0 scale codes
        uint8 [R, C / 32]), one power-of-two scale per 32-element block."""
        a = _c(x, np.float32)
        if a.ndim != 2:
            raise OracleError("mx_quantize expects a 2-D array")
        R, C = a.shape
        q = np.empty((R, C), np.uint8)
        sc = np.empty((R, max(C // 32, 0)), np.uint8)
        rc = self.lib.orc_mx_quantize(_ptr(a), R, C, C, int(fmt), _ptr(q), C, _ptr(sc))
        if rc == -2:
            raise OracleError("the row length must be a multiple of 32")
        if rc == -4:
            raise OracleError("non-finite input")
        return q, sc

    def gemm_mx(self, A, SA, B, SB, alpha=1.0, a_fmt=0, b_fmt=0) -> np.ndarray:
        """C = alpha * sum_b SA[m,b] SB[n,b] sum_{k in b} decA decB (FP64)."""
        A = _c(A, np.uint8)
        B = _c(B, np.uint8)
        SA = _c(SA, np.uint8)
        SB = _c(SB, np.uint8)
        M, K = A.shape
        N = B.shape[0]
        if B.shape[1] != K or K % 32 or SA.shape != (M, K // 32) or SB.shape != (N, K // 32):
            raise OracleError("shape mismatch")
        C = np.empty((M, N), np.float64)
        self.lib.orc_gemm_mx(M, N, K, _ptr(A), K, _ptr(SA), _ptr(B), K, _ptr(SB), float(alpha),
                             int(a_fmt), int(b_fmt), _ptr(C))
        return C

    def max_threads(self) -> int:
        return int(self.lib.orc_max_threads())

    def set_threads(self, n: int) -> None:
        self.lib.orc_set_threads(int(n))


_default = None
_lock = threading.Lock()


def get() -> Oracle:
    """The oracle compiled from ``oracle.c`` (built on first use)."""
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
        return _default


def __getattr__(name):
    # module-level access to the default instance: oracle.gemm(...), etc.
    if name.startswith("_"):
        raise AttributeError(name)
    return getattr(get(), name)
