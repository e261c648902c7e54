"""gemm_fp8_dense_noalloc: the dense FP8 GEMM for callers that may not
allocate device memory (fixed memory budgets planned up front; code running
inside an allocator's callbacks).  Its split-K scratch is a fixed array in
the library's device memory instead of a per-call allocation.

Checked here: the result equals gemm_fp8_dense bit for bit and the oracle
within the FP32 tolerance, on two calls in a row (the second call finds the
first one's leftovers in the array); the call leaves the device's default
memory pool (where cudaMallocAsync draws from) untouched while
gemm_fp8_dense on the same shape grows it, so the shape really needs scratch
and the array served it; a problem whose scratch exceeds the array is
refused with FP8_ERR_SHAPE.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first.  Passes alone in a fresh process and
after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from tests import parity

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 4 << 20              # the array's size, as the header states
RESERVED_MEM_CURRENT = 5             # CUmemPool_attribute values (cuda.h)
USED_MEM_CURRENT = 7


@pytest.fixture(scope="module")
def lib():
    from paper_2602_10262_gb300 import _lib
    return _lib.load()


class DefaultPool:
    """Reserved and used bytes of the current device's default memory pool,
    read through the driver API (the pool cudaMallocAsync allocates from;
    PyTorch's caching allocator does not use it)."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _attr(self, a):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def snapshot(self):
        return self._attr(RESERVED_MEM_CURRENT), self._attr(USED_MEM_CURRENT)


def _plan(lib, M, N, K):
    from paper_2602_10262_gb300 import _lib
    info = _lib.FP8PlanInfo()
    assert lib.gemm_fp8_dense_plan(M, N, K, 0, ctypes.byref(info)) == 0
    return info


def _args(A, B, sa, sb, C, stream):
    M, K = A.shape
    N = B.shape[0]
    st = ctypes.c_void_p(stream.cuda_stream)
    return (M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), sa.data_ptr(), 1,
            sb.data_ptr(), 1, 1.0, C.data_ptr(), C.stride(0), 0, st)


def _operands(M, N, K):
    dev = torch.device("cuda")
    A = workloads.random_codes((M, K), seed=M)
    B = workloads.random_codes((N, K), seed=N)
    sa = (np.abs(workloads.randn_f32((M,), seed=3)) + 0.5).astype(np.float32)
    sb = (np.abs(workloads.randn_f32((N,), seed=4)) + 0.5).astype(np.float32)
    host = (A, B, sa, sb)
    return host, tuple(torch.from_numpy(v).to(dev) for v in host)


def _scratch_shape(t):
    """A product that splits along K and whose slices do not fit a cluster:
    M = 64 rows on the MMA N side (64-wide tiles), K = 8192, and N = 128 t
    rows, i.e. t tiles; with t <= SMs / 8 each tile splits in eight, and
    seven slices' partial sums (7 x 128 x 64 floats, 224 KiB) exceed a CTA's
    ring.  Its scratch: t x 8 x 128 x 64 floats plus 256 bytes of counters."""
    return 64, 128 * t, 8192, t * 8 * 128 * 64 * 4 + 256


def test_noalloc_equals_dense_and_oracle_two_calls(lib, orc):
    sms = lib.fp8_device_sm_count()
    M, N, K, need = _scratch_shape(min(sms // 8, 15))   # 15 tiles: 3.9 MB of the 4 MiB
    assert need <= SCRATCH_BYTES
    info = _plan(lib, M, N, K)
    assert info.splits == 8 and info.cluster == 0 and info.workspace_bytes == need, \
        (info.splits, info.cluster, info.workspace_bytes, need)
    host, (A, B, sa, sb) = _operands(M, N, K)
    pool = DefaultPool()
    ref = torch.empty((M, N), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    s1 = torch.cuda.Stream()
    before = pool.snapshot()
    for i in range(2):                       # the second call reuses the array's old contents
        out = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        assert lib.gemm_fp8_dense_noalloc(*_args(A, B, sa, sb, out, s1)) == 0
        s1.synchronize()
        assert pool.snapshot() == before, "the no-allocation call drew from the default pool"
        if i == 0:
            first = out.clone()
        else:
            assert torch.equal(out, first)
    assert lib.fp8_last_device_error(ctypes.c_void_p(s1.cuda_stream)) == 0

    # control: the regular call on a fresh stream takes its split-K scratch
    # from the default pool, so this shape does need scratch
    s2 = torch.cuda.Stream()
    assert lib.gemm_fp8_dense(*_args(A, B, sa, sb, ref, s2)) == 0
    s2.synchronize()
    after = pool.snapshot()
    assert after[1] >= before[1] + need - 256, (before, after, need)
    assert torch.equal(first, ref), "gemm_fp8_dense_noalloc differs from gemm_fp8_dense"

    Ah, Bh, sah, sbh = host
    parity.check_fp32(first.double().cpu().numpy(), orc.gemm(Ah, Bh, sah, 1, sbh, 1))


@pytest.mark.parametrize("M,N,K", [(16, 4096, 4096), (8, 8192, 4096), (512, 512, 1024)])
def test_noalloc_without_scratch_equals_dense(lib, orc, M, N, K):
    # slices added up within clusters (the first two) or no split at all:
    # no scratch, and the same bits as gemm_fp8_dense
    info = _plan(lib, M, N, K)
    assert info.workspace_bytes == 0 and (info.splits == 1 or info.cluster == info.splits)
    host, (A, B, sa, sb) = _operands(M, N, K)
    st = torch.cuda.current_stream()
    ref = torch.empty((M, N), dtype=torch.float32, device="cuda")
    assert lib.gemm_fp8_dense(*_args(A, B, sa, sb, ref, st)) == 0
    for _ in range(2):
        out = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        assert lib.gemm_fp8_dense_noalloc(*_args(A, B, sa, sb, out, st)) == 0
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    Ah, Bh, sah, sbh = host
    parity.check_fp32(ref.double().cpu().numpy(), orc.gemm(Ah, Bh, sah, 1, sbh, 1))
    assert lib.fp8_last_device_error(ctypes.c_void_p(st.cuda_stream)) == 0


def test_noalloc_rejects_scratch_beyond_the_array(lib):
    sms = lib.fp8_device_sm_count()
    M, N, K, need = _scratch_shape(sms // 8)             # GB300: 19 tiles, 4.98 MB
    if need <= SCRATCH_BYTES:
        pytest.skip(f"{sms} SMs: the largest eight-slice split needs only {need} bytes")
    assert _plan(lib, M, N, K).workspace_bytes == need
    dev = torch.device("cuda")
    A = torch.zeros((M, K), dtype=torch.uint8, device=dev)
    B = torch.zeros((N, K), dtype=torch.uint8, device=dev)
    s = torch.ones(max(M, N), device=dev)
    C = torch.empty((M, N), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    assert lib.gemm_fp8_dense_noalloc(*_args(A, B, s, s, C, st)) == -2
    # the regular entry point takes the same problem from the allocator
    assert lib.gemm_fp8_dense(*_args(A, B, s, s, C, st)) == 0
    torch.cuda.synchronize()
