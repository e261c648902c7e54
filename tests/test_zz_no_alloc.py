"""gemm_fp8_dense_noalloc: the dense FP8 GEMM for callers that may not
allocate device memory (fixed memory budgets planned up front; code running
inside an allocator's callbacks).  Its split-K scratch is a fixed array in
the library's device memory instead of a per-call allocation.

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


@pytest.fixture(scope="module")
def lib():
    from paper_2602_10262_gb300 import _lib
    return _lib.load()


def _args(A, B, sa, sb, C):
    M, K = A.shape
    N = B.shape[0]
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return (M, N, K, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), sa.data_ptr(), 1,
            sb.data_ptr(), 1, 1.0, C.data_ptr(), C.stride(0), 0, st)


@pytest.mark.parametrize("M,N,K", [(16, 4096, 4096), (8, 8192, 4096), (64, 1280, 8192),
                                   (512, 512, 1024)])
def test_noalloc_matches_dense_two_calls(lib, M, N, K):
    # (16, 4096, 4096) and (8, 8192, 4096) split K and add the slices up
    # within clusters (no scratch); (64, 1280, 8192) splits in eight, whose
    # partial sums exceed a CTA's ring, so it goes through the scratch array
    # (2.6 MB); (512, 512, 1024) does not split
    dev = torch.device("cuda")
    A = torch.from_numpy(workloads.random_codes((M, K), seed=M)).to(dev)
    B = torch.from_numpy(workloads.random_codes((N, K), seed=N)).to(dev)
    sa = torch.from_numpy(np.abs(workloads.randn_f32((M,), seed=3)) + 0.5).to(dev)
    sb = torch.from_numpy(np.abs(workloads.randn_f32((N,), seed=4)) + 0.5).to(dev)
    ref = torch.empty((M, N), dtype=torch.float32, device=dev)
    assert lib.gemm_fp8_dense(*_args(A, B, sa, sb, ref)) == 0
    for _ in range(2):                        # the second call reuses the array's old contents
        out = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
        assert lib.gemm_fp8_dense_noalloc(*_args(A, B, sa, sb, out)) == 0
        torch.cuda.synchronize()
        parity.check_fp32(out.double().cpu().numpy(), ref.double().cpu().numpy())
    assert lib.fp8_last_device_error(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0


def test_noalloc_rejects_scratch_beyond_the_array(lib):
    # 19 tiles of 64-wide N split in eight: seven slices' partial sums
    # (224 KB) exceed a CTA's ring, so no cluster; 152 x 128 x 64 floats
    # (4.98 MB) exceed the 4 MiB array -> a clear FP8_ERR_SHAPE, nothing
    # launched
    dev = torch.device("cuda")
    M, N, K = 64, 2432, 8192
    A = torch.zeros((M, K), dtype=torch.uint8, device=dev)
    B = torch.zeros((N, K), dtype=torch.uint8, device=dev)
    s = torch.ones(max(M, N), device=dev)
    C = torch.empty((M, N), dtype=torch.float32, device=dev)
    assert lib.gemm_fp8_dense_noalloc(*_args(A, B, s, s, C)) == -2
    # the regular entry point takes the same problem from the allocator
    assert lib.gemm_fp8_dense(*_args(A, B, s, s, C)) == 0
    torch.cuda.synchronize()
