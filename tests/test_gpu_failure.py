"""GPU tests of the failure path of the GEMM kernel, without a GPU fault.

fp8_test_stall_gemm_loads makes the next launch's TMA producer issue no
operand loads, so the MMA warp's bounded wait for the first stage (a barrier
nothing will complete) runs past a 50 ms limit.  The kernel must then record
FP8_ERR_TIMEOUT in the device error word, stop its other roles, free its
tensor memory and exit with C unwritten; fp8_last_device_error returns the
status and re-zeroes the split-K counters; the next normal launch on the same
operands is bitwise equal to the result taken before the stall.  Covered: a
128-row tile launch, a 256-row tile launch, split-K through a workspace,
split-K within clusters, the 2:4 path and a grouped launch.  Every wait in the
kernel is bounded and the stall only removes loads, so no launch here can
hang or fault.
"""
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

FP8_ERR_TIMEOUT = -7
LIMIT_MS = 50.0


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    yield gb
    gb.fp8_test_stall_gemm_loads(0, 0.0)


def _codes(shape, seed):
    return torch.from_numpy(workloads.small_int_codes(shape, seed=seed)).cuda()


def _dense(gb, M, N, K):
    A, B = _codes((M, K), M + 7), _codes((N, K), N + 11)
    sa = torch.ones(M, device="cuda")
    sb = torch.ones(N, device="cuda")
    return lambda C: gb.gemm_fp8_dense(A, B, sa, 1, sb, 1, 1.0, gb.OUT_F32, C=C)


def _sparse(gb, M, N, K):
    A, B = _codes((M, K), M + 5), _codes((N, K), N + 3)
    vals, meta = gb.prune24_compress(A)
    sa = torch.ones(M, device="cuda")
    sb = torch.ones(N, device="cuda")
    return lambda C: gb.gemm_fp8_sparse24(vals, meta, B, sa, 1, sb, 1, 1.0, gb.OUT_F32, C=C)


def _grouped(gb, M, N, K):
    A1, B1 = _codes((M, K), 21), _codes((N, K), 22)
    A2, B2 = _codes((M // 2, K), 23), _codes((N, K), 24)
    one = torch.ones(max(M, N), device="cuda")
    keep = []

    def run(C):
        C2 = torch.empty((M // 2, N), dtype=torch.float32, device="cuda")
        keep[:] = [C2]
        probs = [gb.make_problem(A1, B1, one, 0, one, 0, C, 1.0, gb.OUT_F32),
                 gb.make_problem(A2, B2, one, 0, one, 0, C2, 1.0, gb.OUT_F32)]
        gb.gemm_fp8_grouped(probs)
    return run


CASES = {
    "128-row tiles": (_dense, 256, 512, 1024),
    "256-row tiles": (_dense, 4096, 4096, 512),
    "split-K workspace": (_dense, 64, 1920, 8192),
    "split-K cluster": (_dense, 16, 4096, 4096),
    "2:4 sparse": (_sparse, 512, 384, 1024),
    "grouped": (_grouped, 512, 768, 512),
}


@pytest.mark.parametrize("name", list(CASES))
def test_stalled_launch_times_out_and_the_next_one_is_exact(gb, name):
    make, M, N, K = CASES[name]
    run = make(gb, M, N, K)
    stream = torch.cuda.Stream()             # a fresh stream: its own split-K workspace
    with torch.cuda.stream(stream):
        ref = torch.empty((M, N), dtype=torch.float32, device="cuda")
        run(ref)
        assert gb.fp8_last_device_error(stream) == 0

        C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        gb.fp8_test_stall_gemm_loads(1, LIMIT_MS)
        try:
            run(C)
            assert gb.fp8_last_device_error(stream) == FP8_ERR_TIMEOUT
        finally:
            gb.fp8_test_stall_gemm_loads(0, 0.0)
        assert torch.isnan(C).all(), "a stalled launch wrote its output"
        assert gb.fp8_last_device_error(stream) == 0     # the word was cleared

        for _ in range(2):                   # the counters and TMEM were left clean
            C.fill_(float("nan"))
            run(C)
            assert gb.fp8_last_device_error(stream) == 0
            assert torch.equal(C, ref)


def test_stall_switch_counts_launches(gb):
    run = _dense(gb, 256, 256, 256)
    ref = torch.empty((256, 256), dtype=torch.float32, device="cuda")
    run(ref)
    assert gb.fp8_last_device_error() == 0
    gb.fp8_test_stall_gemm_loads(2, LIMIT_MS)
    try:
        statuses = []
        for _ in range(3):
            C = torch.full((256, 256), float("nan"), device="cuda")
            run(C)
            statuses.append(gb.fp8_last_device_error())
    finally:
        gb.fp8_test_stall_gemm_loads(0, 0.0)
    assert statuses == [FP8_ERR_TIMEOUT, FP8_ERR_TIMEOUT, 0]
    assert torch.equal(C, ref)
