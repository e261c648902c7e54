"""Python handle for the library's request server (fp8_server_* in the C ABI).

Argument marshalling only: the queues, admission, batching and GPU work live
in csrc/server.cpp.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import torch

from . import _lib

PENDING = 1


class ServerError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.load().fp8_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


@dataclass
class Result:
    status: int
    batch_size: int
    t_submit_us: float
    t_launch_us: float
    t_end_us: float
    t_start_us: float

    @property
    def latency_us(self) -> float:
        return self.t_end_us - self.t_submit_us


def _result(r: _lib.FP8Result) -> Result:
    return Result(r.status, r.batch_size, r.t_submit_us, r.t_launch_us, r.t_end_us, r.t_start_us)


def _check_2d(t, name, dtype, rows, cols, ld) -> None:
    """A tensor passed for a [rows, cols] array with row stride ld must be a
    CUDA tensor of that dtype covering it; raw addresses are not checked."""
    if not isinstance(t, torch.Tensor):
        return
    if not t.is_cuda or t.dtype != dtype or t.dim() != 2:
        raise TypeError(f"{name} must be a 2-D {dtype} CUDA tensor")
    if t.shape[0] < rows or t.shape[1] < cols or (t.numel() > 0 and (t.stride(1) != 1 or t.stride(0) != ld)):
        raise ValueError(f"{name} must cover [{rows}, {cols}] with row stride {ld}, got shape "
                         f"{tuple(t.shape)} and strides {t.stride()}")


def _check_weight(N, K, W, ldw, W_meta, w_scale, w_mode) -> None:
    if W_meta is None:
        _check_2d(W, "W", torch.uint8, N, K, ldw)
    else:
        _check_2d(W, "W", torch.uint8, N, K // 2, K // 2)
        _check_2d(W_meta, "W_meta", torch.uint8, N, (K + 7) // 8, (K + 7) // 8)
    if isinstance(w_scale, torch.Tensor):
        n = N if w_mode else 1
        if not w_scale.is_cuda or w_scale.dtype != torch.float32 or not w_scale.is_contiguous() \
                or w_scale.numel() < n:
            raise ValueError(f"w_scale must be a contiguous float32 CUDA tensor with >= {n} entries")


def overlap_efficiency(results, one_per_interval: bool = True) -> float:
    """Fraction of the GPU's busy time during which two or more batches ran
    at once (the overlap-efficiency metric of the paper, section 3.2).

    Each batch runs within [t_start_us, t_end_us] of its results (requests
    of one batch share the interval and count once).  Busy time is the
    union of the intervals; the concurrent time is where at least two
    intervals cover the clock.  Batches of one tenant share a stream and
    never overlap, so overlap comes from different tenants' streams.  0.0
    when nothing ran.  one_per_interval=False counts identical intervals
    separately (for intervals that are not requests of one batch)."""
    spans = [(r.t_start_us, r.t_end_us) for r in results if r.t_end_us > r.t_start_us]
    if one_per_interval:
        spans = sorted(set(spans))
    events = sorted([(a, 1) for a, _ in spans] + [(b, -1) for _, b in spans],
                    key=lambda e: (e[0], e[1]))
    busy = both = 0.0
    active = 0
    prev = None
    for t, d in events:
        if prev is not None:
            if active >= 1:
                busy += t - prev
            if active >= 2:
                both += t - prev
        active += d
        prev = t
    return both / busy if busy > 0 else 0.0


class Server:
    """fp8_server: continuous batching of FP8 GEMM requests on one GPU, or a
    host-only simulation when ``simulate=(launch_us, us_per_gflop,
    fail_every)`` is given."""

    def __init__(self, num_tenants: int = 2, latency_tenant: int = 0, batching: bool = True,
                 max_batch: int = 0, max_inflight: int = 0, bulk_max_ctas: int = 0,
                 pool_bytes: int = 0, reserve_bytes: int = 0, latency_max_batch: int = 0,
                 latency_max_ctas: int = 0, latency_pool_bytes: int = 0, simulate=None):
        self.lib = _lib.load()
        cfg = _lib.FP8ServerConfig(num_tenants, latency_tenant, int(bool(batching)), max_batch,
                                   max_inflight, bulk_max_ctas, pool_bytes, reserve_bytes,
                                   latency_max_batch, latency_max_ctas, latency_pool_bytes)
        h = ctypes.c_void_p()
        if simulate is None:
            rc = self.lib.fp8_server_create(ctypes.byref(cfg), ctypes.byref(h))
        else:
            launch_us, us_per_gflop, fail_every = simulate
            rc = self.lib.fp8_server_create_simulated(ctypes.byref(cfg), float(launch_us),
                                                      float(us_per_gflop), int(fail_every),
                                                      ctypes.byref(h))
        if rc != 0:
            raise ServerError(rc, "fp8_server_create")
        self.h = h
        self._keep = []
        self._shapes = {}           # handle -> (N, K) of registered weights

    def close(self):
        if self.h:
            self.lib.fp8_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register_weight(self, N: int, K: int, W, w_scale, w_mode: int, W_meta=None,
                        ldw: Optional[int] = None, w_format: int = 0) -> int:
        """W / W_meta / w_scale: CUDA tensors (kept alive by the server object)
        or raw integer device addresses.  w_format: 0 = E4M3, 1 = E5M2 codes."""
        def ptr(t):
            if t is None:
                return None
            if isinstance(t, torch.Tensor):
                self._keep.append(t)
                return t.data_ptr()
            return int(t)
        if ldw is None:
            ldw = W.stride(0) if isinstance(W, torch.Tensor) and W_meta is None else K
        _check_weight(N, K, W, ldw, W_meta, w_scale, w_mode)
        hdl = ctypes.c_uint64()
        rc = self.lib.fp8_server_register_weight_fmt(self.h, N, K, ptr(W), ldw, ptr(W_meta),
                                                     ptr(w_scale), w_mode, int(w_format),
                                                     ctypes.byref(hdl))
        if rc != 0:
            raise ServerError(rc, "fp8_server_register_weight_fmt")
        self._shapes[hdl.value] = (int(N), int(K))
        return hdl.value

    def submit(self, tenant: int, weight: int, M: int, x, ldx: int, out, ldo: int,
               out_dtype: int = 1, alpha: float = 1.0) -> int:
        """x / out: device addresses (int) or CUDA tensors (checked against the
        weight's N and K; the caller keeps them alive until the result)."""
        if weight in self._shapes:
            N, K = self._shapes[weight]
            _check_2d(x, "x", torch.float32, M, K, ldx)
            _check_2d(out, "out", torch.bfloat16 if out_dtype == 1 else torch.float32, M, N, ldo)
        xp = x.data_ptr() if isinstance(x, torch.Tensor) else int(x)
        op = out.data_ptr() if isinstance(out, torch.Tensor) else int(out)
        req = _lib.FP8Request(tenant, weight, M, xp, ldx, op, ldo, out_dtype, alpha)
        t = ctypes.c_uint64()
        rc = self.lib.fp8_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if rc != 0:
            raise ServerError(rc, "fp8_server_submit")
        return t.value

    def poll(self, ticket: int):
        """None while pending, else a Result (status may be an error)."""
        r = _lib.FP8Result()
        rc = self.lib.fp8_server_poll(self.h, ticket, ctypes.byref(r))
        if rc == PENDING:
            return None
        if rc != 0 and r.status == 0:
            raise ServerError(rc, "fp8_server_poll")
        return _result(r)

    def wait(self, ticket: int, timeout_s: float = 30.0):
        r = _lib.FP8Result()
        rc = self.lib.fp8_server_wait(self.h, ticket, ctypes.byref(r), float(timeout_s))
        if rc == PENDING:
            return None
        if rc != 0 and r.status == 0:
            raise ServerError(rc, "fp8_server_wait")
        return _result(r)

    def stats(self) -> dict:
        s = _lib.FP8ServerStats()
        rc = self.lib.fp8_server_get_stats(self.h, ctypes.byref(s))
        if rc != 0:
            raise ServerError(rc, "fp8_server_get_stats")
        return {name: getattr(s, name) for name, _ in s._fields_}

    def now_us(self) -> float:
        return float(self.lib.fp8_server_now_us(self.h))
