"""gb300fp8: FP8 (E4M3 / E5M2) dense and 2:4-sparse GEMM for NVIDIA GB300 (sm_103a).

Thin PyTorch-facing binding over the C ABI of ``libgb300fp8.so``
(include/gb300fp8.h).  Every function has the C entry point's name and only
marshals arguments: it checks dtypes and devices, takes ``data_ptr()`` and
the current CUDA stream, allocates outputs with torch when none are given,
and raises ``Fp8Error`` on a non-zero status.  All arithmetic runs in the
library's CUDA kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import torch

from . import _lib

__all__ = [
    "Fp8Error", "library", "fp8_quantize_e4m3", "fp8_quantize_e5m2", "fp8_quantize_e4m3_prune24", "prune24_compress",
    "prune24_decompress", "gemm_fp8_dense", "gemm_fp8_dense_fmt", "gemm_fp8_sparse24",
    "gemm_fp8_sparse24_fmt", "gemm_fp8_grouped", "gemm_fp8_grouped_ex", "fp8_last_device_error",
    "fp8_device_sm_count", "fp8_test_stall_gemm_loads", "fp8_gemm_set_tile_config", "fp8_gemm_set_multicast",
    "gemm_fp8_grouped_autotune",
    "gemm_fp8_tune_cache_save", "gemm_fp8_tune_cache_load", "gemm_fp8_tune_cache_clear",
    "GroupedGraph", "OUT_F32", "OUT_BF16", "E4M3", "E5M2", "fp8_quantize_mx", "fp8_mx_scales_to_tiled",
    "fp8_mx_scale_tiled_bytes", "gemm_fp8_mx", "gemm_fp8_dense_plan", "gemm_fp8_mx_plan", "gemm_fp8_sparse24_plan",
]

OUT_F32 = 0
OUT_BF16 = 1
E4M3 = 0          # fp8_format values of the C ABI
E5M2 = 1


class Fp8Error(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = library().fp8_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def library():
    """The loaded CDLL (built in tree on first use)."""
    return _lib.load()


def _check(rc: int, where: str):
    if rc != 0:
        raise Fp8Error(rc, where)


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype: torch.dtype, dims: int):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != dims:
        raise ValueError(f"{name} must have {dims} dimensions")
    if dims == 2 and t.numel() > 0 and t.stride(1) != 1:
        raise ValueError(f"{name} must have a contiguous last dimension")


def _shape(t: torch.Tensor, name: str, shape) -> None:
    """An output or companion array must have exactly the extent the call
    writes or reads; a smaller one would be overrun on the device."""
    if tuple(t.shape) != tuple(int(v) for v in shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _packed(t: torch.Tensor, name: str) -> None:
    """Arrays the C ABI takes without a row stride must be contiguous."""
    if t.numel() > 0 and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _scale(t, name: str, n: int) -> None:
    """A scale vector: float32 on the GPU, contiguous, at least n entries."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if not t.is_contiguous() or t.numel() < n:
        raise ValueError(f"{name} must be contiguous with at least {n} entries, got {t.numel()}")


def _ld(t: torch.Tensor) -> int:
    return t.stride(0) if t.dim() == 2 else t.size(-1)


def _p(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def fp8_last_device_error(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device error word."""
    return int(library().fp8_last_device_error(_stream(stream)))


def fp8_device_sm_count() -> int:
    return int(library().fp8_device_sm_count())


def fp8_test_stall_gemm_loads(launches: int, wait_limit_ms: float = 0.0) -> None:
    """Failure-path testing: the next `launches` eager GEMM launches issue no
    operand loads and end with FP8_ERR_TIMEOUT after `wait_limit_ms` (which
    applies to every eager GEMM launch until reset with 0)."""
    _check(library().fp8_test_stall_gemm_loads(int(launches), float(wait_limit_ms)),
           "fp8_test_stall_gemm_loads")


def gemm_fp8_dense_plan(M: int, N: int, K: int, out_dtype: int = OUT_BF16) -> dict:
    """How gemm_fp8_dense would run [M, K] x [N, K]^T now (tile kind, N width,
    k-blocks per stage, K slices, cluster size, grid, operand swap, raster
    band, B multicast group, split-K scratch bytes), without launching."""
    info = _lib.FP8PlanInfo()
    _check(library().gemm_fp8_dense_plan(int(M), int(N), int(K), int(out_dtype), ctypes.byref(info)),
           "gemm_fp8_dense_plan")
    return {name: getattr(info, name) for name, _ in info._fields_}


def gemm_fp8_mx_plan(M: int, N: int, K: int, out_dtype: int = OUT_BF16) -> dict:
    """How gemm_fp8_mx would run [M, K] x [N, K]^T now (fields as
    gemm_fp8_dense_plan), without launching."""
    info = _lib.FP8PlanInfo()
    _check(library().gemm_fp8_mx_plan(int(M), int(N), int(K), int(out_dtype), ctypes.byref(info)),
           "gemm_fp8_mx_plan")
    return {name: getattr(info, name) for name, _ in info._fields_}


def gemm_fp8_sparse24_plan(M: int, N: int, K: int, out_dtype: int = OUT_BF16) -> dict:
    """How gemm_fp8_sparse24 would run a 2:4 [M, K] x [N, K]^T product now
    (fields as gemm_fp8_dense_plan), without launching."""
    info = _lib.FP8PlanInfo()
    _check(library().gemm_fp8_sparse24_plan(int(M), int(N), int(K), int(out_dtype), ctypes.byref(info)),
           "gemm_fp8_sparse24_plan")
    return {name: getattr(info, name) for name, _ in info._fields_}


def fp8_gemm_set_tile_config(mt: int = 0, group_m: int = 0) -> None:
    """Force the GEMM tile shape (mt 1 or 2 row-halves per tile of one CTA,
    3 CTA-pair tiles; raster band height group_m); 0 restores the per-launch
    choice."""
    _check(library().fp8_gemm_set_tile_config(int(mt), int(group_m)), "fp8_gemm_set_tile_config")


def fp8_gemm_set_multicast(mode: int = 0) -> None:
    """B-block multicast within clusters of 128-row-tile launches: 1 where it
    applies, 0 never (default)."""
    _check(library().fp8_gemm_set_multicast(int(mode)), "fp8_gemm_set_multicast")


def _quantize(name: str, x, scale_mode, q, dequant_scale, stream):
    _dev(x, "x", torch.float32, 2)
    R, C = x.shape
    if q is None:
        q = torch.empty((R, C), dtype=torch.uint8, device=x.device)
    if dequant_scale is None:
        dequant_scale = torch.empty((1 if scale_mode == 0 else R,), dtype=torch.float32, device=x.device)
    _dev(q, "q", torch.uint8, 2)
    _shape(q, "q", (R, C))
    _scale(dequant_scale, "dequant_scale", 1 if scale_mode == 0 else R)
    rc = getattr(library(), name)(_p(x), R, C, _ld(x), int(scale_mode), _p(q), _ld(q),
                                  _p(dequant_scale), _stream(stream))
    _check(rc, name)
    return q, dequant_scale


def fp8_quantize_e4m3(x: torch.Tensor, scale_mode: int, q: Optional[torch.Tensor] = None,
                      dequant_scale: Optional[torch.Tensor] = None, stream=None):
    """fp32 [R, C] -> (E4M3 codes uint8 [R, C], dequant scales fp32 [1] or [R])."""
    return _quantize("fp8_quantize_e4m3", x, scale_mode, q, dequant_scale, stream)


def fp8_quantize_e5m2(x: torch.Tensor, scale_mode: int, q: Optional[torch.Tensor] = None,
                      dequant_scale: Optional[torch.Tensor] = None, stream=None):
    """fp32 [R, C] -> (E5M2 codes uint8 [R, C], dequant scales fp32 [1] or [R])."""
    return _quantize("fp8_quantize_e5m2", x, scale_mode, q, dequant_scale, stream)


def fp8_quantize_e4m3_prune24(x: torch.Tensor, q: Optional[torch.Tensor] = None,
                              dequant_scale: Optional[torch.Tensor] = None,
                              a_vals: Optional[torch.Tensor] = None, a_meta: Optional[torch.Tensor] = None,
                              stream=None):
    """fp32 [R, C] (C % 128 == 0) -> (E4M3 codes [R, C], per-row dequant
    scales [R], kept codes [R, C/2], metadata [R, C/8]): per-row
    quantisation and the 2:4 compression of its codes in one pass, bitwise
    fp8_quantize_e4m3(x, 1) followed by prune24_compress."""
    _dev(x, "x", torch.float32, 2)
    R, C = x.shape
    dev = x.device
    if q is None:
        q = torch.empty((R, C), dtype=torch.uint8, device=dev)
    if dequant_scale is None:
        dequant_scale = torch.empty((R,), dtype=torch.float32, device=dev)
    if a_vals is None:
        a_vals = torch.empty((R, C // 2), dtype=torch.uint8, device=dev)
    if a_meta is None:
        a_meta = torch.empty((R, C // 8), dtype=torch.uint8, device=dev)
    _dev(q, "q", torch.uint8, 2)
    _shape(q, "q", (R, C))
    _scale(dequant_scale, "dequant_scale", R)
    for t, nm, shp in ((a_vals, "a_vals", (R, C // 2)), (a_meta, "a_meta", (R, C // 8))):
        _dev(t, nm, torch.uint8, 2)
        _shape(t, nm, shp)
        _packed(t, nm)
    rc = library().fp8_quantize_e4m3_prune24(_p(x), R, C, _ld(x), _p(q), _ld(q), _p(dequant_scale),
                                             _p(a_vals), _p(a_meta), _stream(stream))
    _check(rc, "fp8_quantize_e4m3_prune24")
    return q, dequant_scale, a_vals, a_meta


def fp8_mx_scale_tiled_bytes(rows: int, cols: int) -> int:
    """Bytes of the tiled E8M0 scale layout of a [rows, cols] operand."""
    return int(library().fp8_mx_scale_tiled_bytes(int(rows), int(cols)))


def fp8_quantize_mx(x: torch.Tensor, fmt: int = E4M3, scale_layout: int = 1,
                    q: Optional[torch.Tensor] = None, scales: Optional[torch.Tensor] = None,
                    stream=None):
    """Block-scaled quantisation: fp32 [R, C] (C % 32 == 0) -> (codes uint8
    [R, C], E8M0 scale codes: uint8 [R, C / 32] for scale_layout 0, the tiled
    bytes gemm_fp8_mx reads for scale_layout 1)."""
    _dev(x, "x", torch.float32, 2)
    R, C = x.shape
    if q is None:
        q = torch.empty((R, C), dtype=torch.uint8, device=x.device)
    _dev(q, "q", torch.uint8, 2)
    _shape(q, "q", (R, C))
    if scale_layout == 0:
        shape = (R, C // 32)
    else:
        shape = (fp8_mx_scale_tiled_bytes(R, C),)
    if scales is None:
        scales = torch.empty(shape, dtype=torch.uint8, device=x.device)
    _shape(scales, "scales", shape)
    _packed(scales, "scales")
    rc = library().fp8_quantize_mx(_p(x), R, C, _ld(x), int(fmt), _p(q), _ld(q), _p(scales),
                                   int(scale_layout), _stream(stream))
    _check(rc, "fp8_quantize_mx")
    return q, scales


def fp8_mx_scales_to_tiled(scales: torch.Tensor, rows: int, cols: int,
                           tiled: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Row-major E8M0 scales [rows, cols / 32] -> the tiled layout."""
    _dev(scales, "scales", torch.uint8, 2)
    _shape(scales, "scales", (rows, cols // 32))
    _packed(scales, "scales")
    n = fp8_mx_scale_tiled_bytes(rows, cols)
    if tiled is None:
        tiled = torch.empty((n,), dtype=torch.uint8, device=scales.device)
    _shape(tiled, "tiled", (n,))
    rc = library().fp8_mx_scales_to_tiled(_p(scales), int(rows), int(cols), _p(tiled), _stream(stream))
    _check(rc, "fp8_mx_scales_to_tiled")
    return tiled


def gemm_fp8_mx(A: torch.Tensor, a_scales: torch.Tensor, B: torch.Tensor, b_scales: torch.Tensor,
                alpha: float = 1.0, out_dtype: int = OUT_BF16, a_format: int = E4M3,
                b_format: int = E4M3, C: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Block-scaled GEMM: C[M, N] = alpha * sum_b 2^sa 2^sb dec(A) dec(B)^T over
    32-element blocks; a_scales / b_scales in the tiled layout."""
    _dev(A, "A", torch.uint8, 2)
    _dev(B, "B", torch.uint8, 2)
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("K mismatch")
    for t, nm, rows in ((a_scales, "a_scales", M), (b_scales, "b_scales", N)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8:
            raise TypeError(f"{nm} must be a uint8 CUDA tensor")
        _packed(t, nm)
        if t.numel() < fp8_mx_scale_tiled_bytes(rows, K):
            raise ValueError(f"{nm} must hold {fp8_mx_scale_tiled_bytes(rows, K)} bytes")
    C = _out(C, M, N, out_dtype, A.device)
    rc = library().gemm_fp8_mx(M, N, K, _p(A), _ld(A), _p(a_scales), _p(B), _ld(B), _p(b_scales),
                               float(alpha), _p(C), _ld(C), int(out_dtype), int(a_format), int(b_format),
                               _stream(stream))
    _check(rc, "gemm_fp8_mx")
    return C


def prune24_compress(a: torch.Tensor, a_vals: Optional[torch.Tensor] = None,
                     a_meta: Optional[torch.Tensor] = None, stream=None):
    """E4M3 codes [M, K] -> (kept codes [M, K/2], metadata [M, ceil(K/8)])."""
    _dev(a, "a", torch.uint8, 2)
    M, K = a.shape
    if a_vals is None:
        a_vals = torch.empty((M, K // 2), dtype=torch.uint8, device=a.device)
    if a_meta is None:
        a_meta = torch.empty((M, (K + 7) // 8), dtype=torch.uint8, device=a.device)
    for t, nm, shp in ((a_vals, "a_vals", (M, K // 2)), (a_meta, "a_meta", (M, (K + 7) // 8))):
        _dev(t, nm, torch.uint8, 2)
        _shape(t, nm, shp)
        _packed(t, nm)
    rc = library().prune24_compress(_p(a), M, K, _ld(a), _p(a_vals), _p(a_meta), _stream(stream))
    _check(rc, "prune24_compress")
    return a_vals, a_meta


def prune24_decompress(a_vals: torch.Tensor, a_meta: torch.Tensor, K: int,
                       out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    _dev(a_vals, "a_vals", torch.uint8, 2)
    _dev(a_meta, "a_meta", torch.uint8, 2)
    M = a_vals.shape[0]
    if out is None:
        out = torch.empty((M, K), dtype=torch.uint8, device=a_vals.device)
    for t, nm, shp in ((a_vals, "a_vals", (M, K // 2)), (a_meta, "a_meta", (M, (K + 7) // 8)),
                       (out, "out", (M, K))):
        _dev(t, nm, torch.uint8, 2)
        _shape(t, nm, shp)
        _packed(t, nm)
    rc = library().prune24_decompress(_p(a_vals), _p(a_meta), M, K, _p(out), _stream(stream))
    _check(rc, "prune24_decompress")
    return out


def _out(C, rows, cols, out_dtype, device):
    dt = torch.bfloat16 if out_dtype == OUT_BF16 else torch.float32
    if C is None:
        C = torch.empty((rows, cols), dtype=dt, device=device)
    _dev(C, "C", dt, 2)
    _shape(C, "C", (rows, cols))
    return C


def _scales(a_scale, a_mode, M, b_scale, b_mode, N) -> None:
    _scale(a_scale, "a_scale", M if a_mode else 1)
    _scale(b_scale, "b_scale", N if b_mode else 1)


def _sparse_a(a_vals, a_meta, M, K) -> None:
    _shape(a_meta, "a_meta", (M, (K + 7) // 8))
    _packed(a_vals, "a_vals")
    _packed(a_meta, "a_meta")


def gemm_fp8_dense(A: torch.Tensor, B: torch.Tensor, a_scale: torch.Tensor, a_mode: int,
                   b_scale: torch.Tensor, b_mode: int, alpha: float = 1.0,
                   out_dtype: int = OUT_BF16, C: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
    """C[M, N] = alpha * sa * sb * dec(A)[M, K] @ dec(B)[N, K]^T."""
    _dev(A, "A", torch.uint8, 2)
    _dev(B, "B", torch.uint8, 2)
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("K mismatch")
    C = _out(C, M, N, out_dtype, A.device)
    _scales(a_scale, a_mode, M, b_scale, b_mode, N)
    rc = library().gemm_fp8_dense(M, N, K, _p(A), _ld(A), _p(B), _ld(B), _p(a_scale), int(a_mode),
                                  _p(b_scale), int(b_mode), float(alpha), _p(C), _ld(C),
                                  int(out_dtype), _stream(stream))
    _check(rc, "gemm_fp8_dense")
    return C


def gemm_fp8_dense_fmt(A: torch.Tensor, B: torch.Tensor, a_scale: torch.Tensor, a_mode: int,
                       b_scale: torch.Tensor, b_mode: int, alpha: float = 1.0,
                       out_dtype: int = OUT_BF16, a_format: int = E4M3, b_format: int = E4M3,
                       C: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """gemm_fp8_dense with A's codes read as a_format and B's as b_format."""
    _dev(A, "A", torch.uint8, 2)
    _dev(B, "B", torch.uint8, 2)
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("K mismatch")
    C = _out(C, M, N, out_dtype, A.device)
    _scales(a_scale, a_mode, M, b_scale, b_mode, N)
    rc = library().gemm_fp8_dense_fmt(M, N, K, _p(A), _ld(A), _p(B), _ld(B), _p(a_scale),
                                      int(a_mode), _p(b_scale), int(b_mode), float(alpha), _p(C),
                                      _ld(C), int(out_dtype), int(a_format), int(b_format),
                                      _stream(stream))
    _check(rc, "gemm_fp8_dense_fmt")
    return C


def gemm_fp8_sparse24(a_vals: torch.Tensor, a_meta: torch.Tensor, B: torch.Tensor,
                      a_scale: torch.Tensor, a_mode: int, b_scale: torch.Tensor, b_mode: int,
                      alpha: float = 1.0, out_dtype: int = OUT_BF16, out_transposed: bool = False,
                      C: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Same product with A given as (a_vals [M, K/2], a_meta [M, K/8])."""
    _dev(a_vals, "a_vals", torch.uint8, 2)
    _dev(a_meta, "a_meta", torch.uint8, 2)
    _dev(B, "B", torch.uint8, 2)
    M = a_vals.shape[0]
    K = a_vals.shape[1] * 2
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("K mismatch")
    C = _out(C, N if out_transposed else M, M if out_transposed else N, out_dtype, B.device)
    _scales(a_scale, a_mode, M, b_scale, b_mode, N)
    _sparse_a(a_vals, a_meta, M, K)
    rc = library().gemm_fp8_sparse24(M, N, K, _p(a_vals), _p(a_meta), _p(B), _ld(B), _p(a_scale),
                                     int(a_mode), _p(b_scale), int(b_mode), float(alpha), _p(C),
                                     _ld(C), int(out_dtype), int(bool(out_transposed)),
                                     _stream(stream))
    _check(rc, "gemm_fp8_sparse24")
    return C


def gemm_fp8_sparse24_fmt(a_vals: torch.Tensor, a_meta: torch.Tensor, B: torch.Tensor,
                          a_scale: torch.Tensor, a_mode: int, b_scale: torch.Tensor, b_mode: int,
                          alpha: float = 1.0, out_dtype: int = OUT_BF16,
                          out_transposed: bool = False, a_format: int = E4M3,
                          b_format: int = E4M3, C: Optional[torch.Tensor] = None,
                          stream=None) -> torch.Tensor:
    """gemm_fp8_sparse24 with the kept codes of A read as a_format and B as b_format."""
    _dev(a_vals, "a_vals", torch.uint8, 2)
    _dev(a_meta, "a_meta", torch.uint8, 2)
    _dev(B, "B", torch.uint8, 2)
    M = a_vals.shape[0]
    K = a_vals.shape[1] * 2
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("K mismatch")
    C = _out(C, N if out_transposed else M, M if out_transposed else N, out_dtype, B.device)
    _scales(a_scale, a_mode, M, b_scale, b_mode, N)
    _sparse_a(a_vals, a_meta, M, K)
    rc = library().gemm_fp8_sparse24_fmt(M, N, K, _p(a_vals), _p(a_meta), _p(B), _ld(B),
                                         _p(a_scale), int(a_mode), _p(b_scale), int(b_mode),
                                         float(alpha), _p(C), _ld(C), int(out_dtype),
                                         int(bool(out_transposed)), int(a_format), int(b_format),
                                         _stream(stream))
    _check(rc, "gemm_fp8_sparse24_fmt")
    return C


def make_problem(A: torch.Tensor, B: torch.Tensor, a_scale, a_mode, b_scale, b_mode, C,
                 alpha: float = 1.0, out_dtype: int = OUT_BF16, A_meta=None, K: Optional[int] = None,
                 out_transposed: bool = False, a_format: int = E4M3,
                 b_format: int = E4M3) -> _lib.FP8Problem:
    """Build one ``fp8_gemm_problem`` entry (tensors must outlive the call)."""
    sparse = A_meta is not None
    _dev(A, "A", torch.uint8, 2)
    _dev(B, "B", torch.uint8, 2)
    M = A.shape[0]
    N = B.shape[0]
    Kd = A.shape[1] * 2 if sparse else A.shape[1]
    if (K is not None and K != Kd) or B.shape[1] != Kd:
        raise ValueError("K mismatch")
    if sparse:
        _dev(A_meta, "A_meta", torch.uint8, 2)
        _sparse_a(A, A_meta, M, Kd)
    dt = torch.bfloat16 if out_dtype == OUT_BF16 else torch.float32
    _dev(C, "C", dt, 2)
    _shape(C, "C", (N, M) if out_transposed else (M, N))
    _scales(a_scale, a_mode, M, b_scale, b_mode, N)
    return _lib.FP8Problem(M, B.shape[0], Kd, A.data_ptr(), 0 if A_meta is None else A_meta.data_ptr(),
                           _ld(A), B.data_ptr(), _ld(B), a_scale.data_ptr(), int(a_mode),
                           b_scale.data_ptr(), int(b_mode), float(alpha), C.data_ptr(), _ld(C),
                           int(out_dtype), int(bool(out_transposed)), int(a_format),
                           int(b_format))


def gemm_fp8_grouped(problems: Sequence[_lib.FP8Problem], stream=None) -> None:
    """Run every problem in one persistent launch."""
    arr = (_lib.FP8Problem * len(problems))(*problems)
    rc = library().gemm_fp8_grouped(arr, len(problems), _stream(stream))
    _check(rc, "gemm_fp8_grouped")


def gemm_fp8_grouped_ex(problems: Sequence[_lib.FP8Problem], max_ctas: int = 0,
                        stream=None) -> None:
    """gemm_fp8_grouped with the persistent grid capped at max_ctas CTAs
    (0: every SM)."""
    arr = (_lib.FP8Problem * len(problems))(*problems)
    rc = library().gemm_fp8_grouped_ex(arr, len(problems), int(max_ctas), _stream(stream))
    _check(rc, "gemm_fp8_grouped_ex")


def gemm_fp8_grouped_autotune(problems: Sequence[_lib.FP8Problem], max_ctas: int = 0,
                              iters: int = 3, stream=None) -> dict:
    """Time every tile configuration for this problem list, cache the fastest
    and return it as {"mt", "group_m", "ms_per_launch", "bn_max"}."""
    arr = (_lib.FP8Problem * len(problems))(*problems)
    best = _lib.FP8TileConfig()
    rc = library().gemm_fp8_grouped_autotune(arr, len(problems), int(max_ctas), int(iters),
                                             _stream(stream), ctypes.byref(best))
    _check(rc, "gemm_fp8_grouped_autotune")
    return {"mt": best.mt, "group_m": best.group_m, "ms_per_launch": best.ms_per_launch,
            "bn_max": best.bn_max}


def gemm_fp8_tune_cache_save(path: str) -> None:
    _check(library().gemm_fp8_tune_cache_save(path.encode()), "gemm_fp8_tune_cache_save")


def gemm_fp8_tune_cache_load(path: str) -> None:
    _check(library().gemm_fp8_tune_cache_load(path.encode()), "gemm_fp8_tune_cache_load")


def gemm_fp8_tune_cache_clear() -> None:
    _check(library().gemm_fp8_tune_cache_clear(), "gemm_fp8_tune_cache_clear")


class GroupedGraph:
    """A grouped launch captured as a CUDA graph (gemm_fp8_grouped_graph_*)."""

    def __init__(self, problems: Sequence[_lib.FP8Problem], max_ctas: int = 0):
        self.lib = library()
        arr = (_lib.FP8Problem * len(problems))(*problems)
        h = ctypes.c_void_p()
        _check(self.lib.gemm_fp8_grouped_graph_create(arr, len(problems), int(max_ctas),
                                                      ctypes.byref(h)), "gemm_fp8_grouped_graph_create")
        self.h = h

    def update(self, problems: Sequence[_lib.FP8Problem]) -> None:
        arr = (_lib.FP8Problem * len(problems))(*problems)
        _check(self.lib.gemm_fp8_grouped_graph_update(self.h, arr, len(problems)),
               "gemm_fp8_grouped_graph_update")

    def launch(self, stream=None) -> None:
        _check(self.lib.gemm_fp8_grouped_graph_launch(self.h, _stream(stream)),
               "gemm_fp8_grouped_graph_launch")

    def close(self) -> None:
        if self.h:
            self.lib.gemm_fp8_grouped_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
