"""GPU parity of the CTA-pair GEMM tiles (tcgen05 cta_group::2).

A 256 x 256 tile runs on a cluster of two CTAs: each loads 128 rows of A and
128 rows of B, the even CTA issues the pair's MMAs, each CTA stores its half
of the tile.  The tests force the pair tiles (fp8_gemm_set_tile_config(3)),
check through gemm_fp8_dense_plan that the launch really uses them, and
compare with the oracle (small-integer inputs bit for bit, N(0,1) inputs on
sampled entries) and bitwise with the single-CTA 256-row tiles, which sum
each entry in the same order.  Every wait runs with a 500 ms limit here, so
a pipeline that never completes would show as FP8_ERR_TIMEOUT.
"""
import numpy as np
import pytest
import torch

import workloads
from tests import parity, sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


@pytest.fixture
def pair(gb):
    gb.fp8_gemm_set_tile_config(3, 0)
    gb.fp8_test_stall_gemm_loads(0, 500.0)
    yield
    gb.fp8_gemm_set_tile_config(0, 0)
    gb.fp8_test_stall_gemm_loads(0, 0.0)


SHAPES = [(2048, 2560, 1024), (1000, 3000, 640), (4096, 4096, 512), (2304, 2304, 4224)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_pair_tiles_are_planned(gb, pair, M, N, K):
    info = gb.gemm_fp8_dense_plan(M, N, K)
    assert info["mt"] == 3 and info["cluster"] == 2 and info["bn"] == 256, info
    assert info["grid"] % 2 == 0 and info["workspace_bytes"] == 0 and info["splits"] == 1


def _ones(n):
    return torch.ones(n, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_pair_small_integers_bit_exact(gb, orc, pair, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + 1)
    B = workloads.small_int_codes((N, K), seed=N + 2)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = gb.gemm_fp8_dense(At, Bt, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    ref = orc.gemm(A, B, np.ones(1, np.float32), 0, np.ones(1, np.float32), 0)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
    gb.fp8_gemm_set_tile_config(2, 0)                     # single-CTA 256-row tiles
    C2 = gb.gemm_fp8_dense(At, Bt, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32)
    torch.cuda.synchronize()
    assert torch.equal(C, C2)


@pytest.mark.parametrize("out_dtype", [0, 1])
def test_pair_normal_inputs_sampled(gb, orc, pair, out_dtype):
    M, N, K = 4096, 4096, 4096
    x = workloads.randn_f32((M, K), seed=71)
    w = workloads.randn_f32((N, K), seed=72)
    A, dA = gb.fp8_quantize_e4m3(torch.from_numpy(x).cuda(), 1)
    B, dB = gb.fp8_quantize_e4m3(torch.from_numpy(w).cuda(), 1)
    C = gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 0.5, out_dtype)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    ms, ns = sampled.entries(M, N, seed=73)
    ref, S = sampled.reference(orc, x, w, ms, ns, alpha=0.5)
    got = C[torch.from_numpy(ms).cuda(), torch.from_numpy(ns).cuda()].float().cpu().numpy()
    if out_dtype:
        parity.check_bf16(got, ref, S, K)
    else:
        parity.check_fp32(got, ref)


def test_pair_grouped_equals_single_cta_tiles(gb, orc, pair):
    shapes = [(2048, 2048, 1024), (1536, 4096, 512), (1024, 2560, 2048)]
    probs, outs, keep = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        A, dA = orc.quantize(workloads.randn_f32((M, K), seed=80 + i), 1)
        B, dB = orc.quantize(workloads.randn_f32((N, K), seed=90 + i), 1)
        t = [torch.from_numpy(v).cuda() for v in (A, B, dA, dB)]
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        keep += t
        outs.append(C)
        probs.append(gb.make_problem(t[0], t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16))
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    got = [c.clone() for c in outs]
    gb.fp8_gemm_set_tile_config(2, 0)
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    for a, b in zip(got, outs):
        assert torch.equal(a, b)


def test_pair_stalled_launch_times_out(gb, pair):
    M, N, K = 2048, 2560, 1024
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


def test_pair_raster_band(gb):
    """CTA-pair launches whose operands exceed L2 walk 8-row raster bands
    (fewer HBM re-reads per wave of 76 tiles), others 16; a forced band
    stands."""
    gb.fp8_gemm_set_tile_config(0, 0)
    big = gb.gemm_fp8_dense_plan(16384, 16384, 16384)
    assert big["mt"] == 3 and big["group_m"] == 8
    mid = gb.gemm_fp8_dense_plan(4096, 4096, 4096)
    assert mid["mt"] == 3 and mid["group_m"] == 16
    assert gb.gemm_fp8_dense_plan(1024, 1024, 1024)["group_m"] == 16
    gb.fp8_gemm_set_tile_config(3, 4)
    try:
        assert gb.gemm_fp8_dense_plan(16384, 16384, 16384)["group_m"] == 4
    finally:
        gb.fp8_gemm_set_tile_config(0, 0)


def test_pair_grouped_graph_equals_direct(gb, orc, pair):
    """A CUDA-graph grouped launch of CTA-pair tiles (the kernel node carries
    the cluster shape) equals the direct launch bit for bit, before and after
    a pointer update.  A node without clusters would do no work and record
    FP8_ERR_UNSUPPORTED, so both checks would fail."""
    shapes = [(2048, 2048, 1024), (1536, 4096, 512), (1024, 2560, 2048)]

    def problems(seed):
        probs, outs, keep = [], [], []
        for i, (M, N, K) in enumerate(shapes):
            A, dA = orc.quantize(workloads.randn_f32((M, K), seed=seed + i), 1)
            B, dB = orc.quantize(workloads.randn_f32((N, K), seed=seed + 10 + i), 1)
            t = [torch.from_numpy(v).cuda() for v in (A, B, dA, dB)]
            C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
            keep += t
            outs.append(C)
            probs.append(gb.make_problem(t[0], t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16))
        return probs, outs, keep

    p1, o1, k1 = problems(300)
    p2, o2, k2 = problems(400)
    gb.gemm_fp8_grouped(p1)
    gb.gemm_fp8_grouped(p2)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    ref1, ref2 = [c.clone() for c in o1], [c.clone() for c in o2]
    for c in o1 + o2:
        c.zero_()
    g = gb.GroupedGraph(p1)
    g.launch()
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    for a, b in zip(ref1, o1):
        assert torch.equal(a, b)
    g.update(p2)
    g.launch()
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    for a, b in zip(ref2, o2):
        assert torch.equal(a, b)
    g.close()


def test_pair_chosen_for_long_k_mid_rows(gb):
    """Pairs where they occupy as many SMs as 128-row tiles and K >= 4096;
    128-row tiles at the same shape with short K."""
    gb.fp8_gemm_set_tile_config(0, 0)
    assert gb.gemm_fp8_dense_plan(512, 8192, 8192)["mt"] == 3
    assert gb.gemm_fp8_dense_plan(2048, 2048, 2048)["mt"] == 1
    assert gb.gemm_fp8_dense_plan(256, 8192, 8192)["mt"] == 1


def test_single_cta_cap_takes_no_pairs(gb, orc):
    """A launch capped at one CTA runs 128-row tiles (a pair needs two CTAs)
    and gives the bits of the uncapped pair launch."""
    gb.fp8_gemm_set_tile_config(0, 0)
    M, N, K = 2048, 2560, 1024
    A, dA = orc.quantize(workloads.randn_f32((M, K), seed=31), 1)
    B, dB = orc.quantize(workloads.randn_f32((N, K), seed=32), 1)
    t = [torch.from_numpy(v).cuda() for v in (A, B, dA, dB)]
    outs = []
    for cap in (0, 1, 2):
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        gb.gemm_fp8_grouped_ex([gb.make_problem(t[0], t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16)], cap)
        torch.cuda.synchronize()
        assert gb.fp8_last_device_error() == 0
        outs.append(C)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
