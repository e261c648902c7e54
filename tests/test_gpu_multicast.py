"""GPU tests of B-block multicast within clusters (fp8_gemm_set_multicast(1);
off by default).

Launches of 128-row tiles of one dense, unsplit problem run as clusters of
4 (or 2) CTAs on consecutive row blocks of one N column; each CTA loads a
quarter (half) of the shared B block per stage and multicasts it to the
cluster.  The MMAs and their order are those of the launch without
multicast, so the tests compare the two bit for bit (ragged edges, an odd
number of k-blocks, the swapped skinny orientation), small-integer inputs
against the oracle exactly, and drive the timeout path with the loads
withheld.  Every wait runs with a 500 ms limit here.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


@pytest.fixture
def limits(gb):
    gb.fp8_gemm_set_tile_config(0, 0)
    gb.fp8_gemm_set_multicast(1)
    gb.fp8_test_stall_gemm_loads(0, 500.0)
    yield
    gb.fp8_gemm_set_multicast(0)
    gb.fp8_test_stall_gemm_loads(0, 0.0)


def _ones(n):
    return torch.ones(n, dtype=torch.float32, device="cuda")


# (M, N, K): square mid-size, 256-wide tiles, ragged edges, an odd number of
# k-blocks, the swapped skinny orientation (B side = the 128 activation rows)
SHAPES = [(1024, 1024, 1024), (2048, 2048, 2048), (1000, 1000, 1152), (1024, 768, 640), (128, 8192, 4096)]


def test_multicast_is_planned(gb, limits):
    info = gb.gemm_fp8_dense_plan(1024, 1024, 1024)
    assert info["mt"] == 1 and info["multicast"] in (2, 4), info
    assert info["cluster"] == info["multicast"] and info["grid"] % info["multicast"] == 0
    gb.fp8_gemm_set_multicast(0)
    info = gb.gemm_fp8_dense_plan(1024, 1024, 1024)
    assert info["multicast"] == 0 and info["cluster"] == 0
    gb.fp8_gemm_set_multicast(1)
    # split-K and CTA-pair launches take no multicast
    assert gb.gemm_fp8_dense_plan(16, 8192, 8192)["multicast"] == 0
    assert gb.gemm_fp8_dense_plan(8192, 8192, 8192)["multicast"] == 0
    with pytest.raises(gb.Fp8Error):
        gb.fp8_gemm_set_multicast(2)


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_multicast_equals_plain_launch(gb, limits, M, N, K):
    info = gb.gemm_fp8_dense_plan(M, N, K)
    assert info["multicast"] > 0, info
    x = workloads.randn_f32((M, K), seed=M + 5)
    w = workloads.randn_f32((N, K), seed=N + 6)
    A, dA = gb.fp8_quantize_e4m3(torch.from_numpy(x).cuda(), 1)
    B, dB = gb.fp8_quantize_e4m3(torch.from_numpy(w).cuda(), 1)
    for out in (gb.OUT_BF16, gb.OUT_F32):
        C1 = gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 0.75, out)
        torch.cuda.synchronize()
        assert gb.fp8_last_device_error() == 0
        gb.fp8_gemm_set_multicast(0)
        C0 = gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 0.75, out)
        torch.cuda.synchronize()
        gb.fp8_gemm_set_multicast(1)
        assert gb.fp8_last_device_error() == 0
        assert torch.equal(C0, C1)


@pytest.mark.parametrize("M,N,K", [(1024, 1024, 1024), (1000, 1000, 1152), (128, 8192, 4096)])
def test_multicast_small_integers_bit_exact(gb, orc, limits, M, N, K):
    assert gb.gemm_fp8_dense_plan(M, N, K)["multicast"] > 0
    A = workloads.small_int_codes((M, K), seed=M + 1)
    B = workloads.small_int_codes((N, K), seed=N + 2)
    C = gb.gemm_fp8_dense(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), _ones(1), 0, _ones(1), 0,
                          1.0, gb.OUT_F32)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    ref = orc.gemm(A, B, np.ones(1, np.float32), 0, np.ones(1, np.float32), 0)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)


def test_multicast_grouped_graph_equals_direct(gb, limits):
    """A one-problem CUDA-graph launch carries the cluster shape too."""
    M, N, K = 1024, 1024, 1024
    At = torch.from_numpy(workloads.small_int_codes((M, K), seed=9)).cuda()
    Bt = torch.from_numpy(workloads.small_int_codes((N, K), seed=10)).cuda()
    ref = gb.gemm_fp8_dense(At, Bt, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_BF16)
    C = torch.zeros_like(ref)
    g = gb.GroupedGraph([gb.make_problem(At, Bt, _ones(1), 0, _ones(1), 0, C, 1.0, gb.OUT_BF16)])
    g.launch()
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    assert torch.equal(C, ref)
    g.close()


def test_multicast_stalled_launch_times_out(gb, limits):
    M, N, K = 1024, 1024, 1024
    At = torch.from_numpy(workloads.small_int_codes((M, K), seed=5)).cuda()
    Bt = torch.from_numpy(workloads.small_int_codes((N, K), seed=6)).cuda()
    ref = gb.gemm_fp8_dense(At, Bt, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32)
    assert gb.fp8_last_device_error() == 0
    C = torch.full((M, N), float("nan"), device="cuda")
    gb.fp8_test_stall_gemm_loads(1, 50.0)
    try:
        gb.gemm_fp8_dense(At, Bt, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32, C=C)
        assert gb.fp8_last_device_error() == -7
    finally:
        gb.fp8_test_stall_gemm_loads(0, 500.0)
    assert torch.isnan(C).all()
    gb.gemm_fp8_dense(At, Bt, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32, C=C)
    assert gb.fp8_last_device_error() == 0
    assert torch.equal(C, ref)


def test_multicast_off_by_default(gb):
    """A fresh process plans no multicast until it is switched on."""
    code = ("import paper_2602_10262_gb300 as gb; gb.library(); "
            "print(gb.gemm_fp8_dense_plan(1024, 1024, 1024)['multicast'])")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "0"
