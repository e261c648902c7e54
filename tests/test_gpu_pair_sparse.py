"""GPU parity of the 2:4-sparse CTA-pair tiles (tcgen05.mma.sp cta_group::2).

A 256 x 224 tile runs on a cluster of two CTAs: each loads the kept codes and
metadata of its 128 rows of A and 112 rows of B, copies its metadata into
its own tensor memory, the even CTA issues the pair's sparse MMAs, and each
CTA stores its half of the tile from one of two accumulators.  The tests
force the pair tiles (fp8_gemm_set_tile_config(3)), check through
gemm_fp8_sparse24_plan that the launch uses them, and compare with the
oracle (small-integer inputs bit for bit, N(0,1) inputs on sampled entries
within the parity bounds) and bitwise with the one-CTA tiles, which sum each
entry over the same logical K = 64 steps in the same order.  Every wait runs
with a 500 ms limit here.
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ones(n):
    return torch.ones(n, dtype=torch.float32, device="cuda")


# several pair tiles in both directions; ragged rows (the odd CTA's half past
# A's end) and ragged columns (a last tile 88 wide: the odd CTA's B rows all
# past B's end); an odd number of k-blocks (the last stage half empty)
SHAPES = [(2048, 2560, 1024), (1000, 3000, 640), (4096, 4096, 512), (2304, 2304, 4224)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_sparse_pair_tiles_are_planned(gb, pair, M, N, K):
    info = gb.gemm_fp8_sparse24_plan(M, N, K)
    assert info["mt"] == 3 and info["cluster"] == 2 and info["bn"] == 224, info
    assert info["grid"] % 2 == 0 and info["splits"] == 1 and info["workspace_bytes"] == 0
    assert info["k_blocks_per_stage"] == 2 and info["swapped"] == 0


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_sparse_pair_small_integers_bit_exact(gb, orc, pair, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + 31)
    B = workloads.small_int_codes((N, K), seed=N + 32)
    vals, meta = orc.prune24(A)
    tv, tm, tB = _cuda(vals), _cuda(meta), _cuda(B)
    C = gb.gemm_fp8_sparse24(tv, tm, tB, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    one = np.ones(1, np.float32)
    ref = orc.gemm_sparse24(vals, meta, B, K, one, 0, one, 0)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)
    for mt in (2, 1):                                    # one-CTA tiles, same sums
        gb.fp8_gemm_set_tile_config(mt, 0)
        C2 = gb.gemm_fp8_sparse24(tv, tm, tB, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32)
        torch.cuda.synchronize()
        assert gb.fp8_last_device_error() == 0
        assert torch.equal(C, C2), mt


@pytest.mark.parametrize("out_dtype", [0, 1])
def test_sparse_pair_normal_inputs_sampled(gb, orc, pair, out_dtype):
    M, N, K = 4096, 4096, 4096
    x = workloads.randn_f32((M, K), seed=171)
    w = workloads.randn_f32((N, K), seed=172)
    A, dA = orc.quantize(x, 1)
    B, dB = orc.quantize(w, 1)
    vals, meta = orc.prune24(A)
    tv, tm, tB, tdA, tdB = _cuda(vals), _cuda(meta), _cuda(B), _cuda(dA), _cuda(dB)
    C = gb.gemm_fp8_sparse24(tv, tm, tB, tdA, 1, tdB, 1, 0.5, out_dtype)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    Ap = orc.decompress24(vals, meta, K)
    ms, ns = sampled.entries(M, N, seed=173)
    ref = orc.gemm_sampled(Ap, B, dA, 1, dB, 1, 0.5, ms, ns)
    S = orc.gemm_sampled(parity.abs_codes(Ap), parity.abs_codes(B), dA, 1, dB, 1, 0.5, ms, ns)
    got = C[torch.from_numpy(ms).cuda(), torch.from_numpy(ns).cuda()].float().cpu().numpy()
    if out_dtype:
        parity.check_bf16(got, ref, S, K)
    else:
        parity.check_fp32(got, ref)
    gb.fp8_gemm_set_tile_config(2, 0)
    C2 = gb.gemm_fp8_sparse24(tv, tm, tB, tdA, 1, tdB, 1, 0.5, out_dtype)
    torch.cuda.synchronize()
    assert torch.equal(C, C2)


def test_sparse_pair_transposed_output(gb, orc, pair):
    M, N, K = 1000, 3000, 640
    A = workloads.small_int_codes((M, K), seed=41)
    B = workloads.small_int_codes((N, K), seed=42)
    vals, meta = orc.prune24(A)
    tv, tm, tB = _cuda(vals), _cuda(meta), _cuda(B)
    Ct = gb.gemm_fp8_sparse24(tv, tm, tB, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_BF16, True)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    gb.fp8_gemm_set_tile_config(2, 0)
    C = gb.gemm_fp8_sparse24(tv, tm, tB, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_BF16)
    torch.cuda.synchronize()
    assert torch.equal(Ct.T, C)


def test_sparse_pair_grouped_equals_single_cta_tiles(gb, orc, pair):
    shapes = [(2048, 2048, 1024), (1536, 4096, 512), (1024, 2560, 2048)]
    probs, outs, keep = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        A, dA = orc.quantize(workloads.randn_f32((M, K), seed=180 + i), 1)
        B, dB = orc.quantize(workloads.randn_f32((N, K), seed=190 + i), 1)
        vals, meta = orc.prune24(A)
        t = [_cuda(v) for v in (vals, meta, B, dA, dB)]
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        keep += t
        outs.append(C)
        probs.append(gb.make_problem(t[0], t[2], t[3], 1, t[4], 1, C, 1.0, gb.OUT_BF16, A_meta=t[1]))
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    got = [c.clone() for c in outs]
    gb.fp8_gemm_set_tile_config(2, 0)
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    for a, b in zip(got, outs):
        assert torch.equal(a, b)


def test_sparse_pair_stalled_launch_times_out(gb, orc, pair):
    M, N, K = 2048, 2560, 1024
    A = workloads.small_int_codes((M, K), seed=55)
    B = workloads.small_int_codes((N, K), seed=56)
    vals, meta = orc.prune24(A)
    tv, tm, tB = _cuda(vals), _cuda(meta), _cuda(B)
    ref = gb.gemm_fp8_sparse24(tv, tm, tB, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32)
    assert gb.fp8_last_device_error() == 0
    C = torch.full((M, N), float("nan"), device="cuda")
    gb.fp8_test_stall_gemm_loads(1, 50.0)
    try:
        gb.gemm_fp8_sparse24(tv, tm, tB, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32, C=C)
        assert gb.fp8_last_device_error() == -7
    finally:
        gb.fp8_test_stall_gemm_loads(0, 500.0)
    assert torch.isnan(C).all()
    gb.gemm_fp8_sparse24(tv, tm, tB, _ones(1), 0, _ones(1), 0, 1.0, gb.OUT_F32, C=C)
    assert gb.fp8_last_device_error() == 0
    assert torch.equal(C, ref)


def test_sparse_narrow_tiles_take_no_pairs(gb, pair):
    """Forced pairs fall back where they do not apply: N tiles under 224."""
    info = gb.gemm_fp8_sparse24_plan(2048, 200, 1024)
    assert info["mt"] != 3 and info["cluster"] == 0, info


def test_sparse_pair_raster_band(gb):
    """2:4 pair launches keep 16-row raster bands even beyond L2 (their A
    rows are 0.625 of the dense bytes); dense pairs there take 8."""
    assert gb.gemm_fp8_sparse24_plan(16384, 16384, 16384)["mt"] == 3
    assert gb.gemm_fp8_sparse24_plan(16384, 16384, 16384)["group_m"] == 16
    assert gb.gemm_fp8_dense_plan(16384, 16384, 16384)["group_m"] == 8


def test_grouped_list_split_by_tile_kind_equals_singles(gb, orc):
    """A list mixing large dense and 2:4 problems (CTA-pair tiles alone) with
    small ones runs as separate launches per tile kind; every output equals
    the problem issued alone, bit for bit, and forcing one kind for the
    whole list changes nothing either."""
    shapes = [(2048, 2560, 1024, False), (4096, 2048, 1024, True), (64, 512, 256, False),
              (300, 200, 512, True), (1024, 4096, 2048, False)]
    probs, outs, singles, keep = [], [], [], []
    for i, (M, N, K, sparse) in enumerate(shapes):
        A, dA = orc.quantize(workloads.randn_f32((M, K), seed=300 + i), 1)
        B, dB = orc.quantize(workloads.randn_f32((N, K), seed=310 + i), 1)
        tB, tdA, tdB = _cuda(B), _cuda(dA), _cuda(dB)
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        if sparse:
            vals, meta = orc.prune24(A)
            tv, tm = _cuda(vals), _cuda(meta)
            probs.append(gb.make_problem(tv, tB, tdA, 1, tdB, 1, C, 1.0, gb.OUT_BF16, A_meta=tm))
            singles.append(gb.gemm_fp8_sparse24(tv, tm, tB, tdA, 1, tdB, 1, 1.0, gb.OUT_BF16))
            keep += [tv, tm]
        else:
            tA = _cuda(A)
            probs.append(gb.make_problem(tA, tB, tdA, 1, tdB, 1, C, 1.0, gb.OUT_BF16))
            singles.append(gb.gemm_fp8_dense(tA, tB, tdA, 1, tdB, 1, 1.0, gb.OUT_BF16))
            keep.append(tA)
        keep += [tB, tdA, tdB]
        outs.append(C)
    assert gb.gemm_fp8_dense_plan(2048, 2560, 1024)["mt"] == 3
    assert gb.gemm_fp8_sparse24_plan(4096, 2048, 1024)["mt"] == 3
    assert gb.gemm_fp8_dense_plan(1024, 4096, 2048)["mt"] == 1
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    for i, (C, Cs) in enumerate(zip(outs, singles)):
        assert torch.equal(C, Cs), i
    try:
        gb.fp8_gemm_set_tile_config(1, 0)
        for C in outs:
            C.zero_()
        gb.gemm_fp8_grouped_ex(probs, 136)
        torch.cuda.synchronize()
        assert gb.fp8_last_device_error() == 0
    finally:
        gb.fp8_gemm_set_tile_config(0, 0)
    for i, (C, Cs) in enumerate(zip(outs, singles)):
        assert torch.equal(C, Cs), i
