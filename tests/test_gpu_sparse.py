"""GPU parity: gemm_fp8_sparse24 against the FP64 oracle (sparse GEMM equals
the dense GEMM of the decompressed pruned A, paper section 6)."""
import numpy as np
import pytest
import torch

import workloads
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sparse(gb, vals, meta, B, dA, a_mode, dB, b_mode, alpha, out_dtype, out_transposed=False):
    C = gb.gemm_fp8_sparse24(_cuda(vals), _cuda(meta), _cuda(B), _cuda(dA), a_mode, _cuda(dB),
                             b_mode, alpha, out_dtype, out_transposed)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    return C.float().cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 128), (256, 256, 256), (200, 72, 384),
                                   (16, 512, 1024), (300, 17, 4096)])
def test_small_integers_bit_exact(gb, orc, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + 7)
    B = workloads.small_int_codes((N, K), seed=N + 8)
    vals, meta = orc.prune24(A)
    one = np.ones(1, np.float32)
    C = _sparse(gb, vals, meta, B, one, 0, one, 0, 1.0, gb.OUT_F32)
    ref = orc.gemm_sparse24(vals, meta, B, K, one, 0, one, 0)
    assert np.array_equal(C.astype(np.float64), ref)


def _pruned(M, N, K, orc, seed):
    x = workloads.randn_f32((M, K), seed=workloads.SEED_A + seed)
    w = workloads.randn_f32((N, K), seed=workloads.SEED_B + seed)
    A, dA = orc.quantize(x, 1)
    B, dB = orc.quantize(w, 1)
    vals, meta = orc.prune24(A)
    return vals, meta, dA, B, dB


def test_sparse_256_fp32(gb, orc):
    vals, meta, dA, B, dB = _pruned(256, 256, 256, orc, 0)
    C = _sparse(gb, vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_F32)
    parity.check_fp32(C, orc.gemm_sparse24(vals, meta, B, 256, dA, 1, dB, 1))


@pytest.mark.parametrize("M,N,K", [(1024, 1024, 1024), (1000, 700, 512), (128, 2048, 2048),
                                   (2048, 2048, 2048)])
def test_sparse_bf16(gb, orc, M, N, K):
    vals, meta, dA, B, dB = _pruned(M, N, K, orc, M)
    C = _sparse(gb, vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16)
    ref = orc.gemm_sparse24(vals, meta, B, K, dA, 1, dB, 1)
    S = orc.gemm_sparse24(parity.abs_codes(vals), meta, parity.abs_codes(B), K, dA, 1, dB, 1)
    parity.check_bf16(C, ref, S, K)


def test_sparse_transposed_output(gb, orc):
    vals, meta, dA, B, dB = _pruned(384, 200, 512, orc, 5)
    C = _sparse(gb, vals, meta, B, dA, 1, dB, 1, 0.5, gb.OUT_F32, out_transposed=True)
    assert C.shape == (200, 384)
    parity.check_fp32(C.T, orc.gemm_sparse24(vals, meta, B, 512, dA, 1, dB, 1, 0.5))


def test_sparse_full_size_sampled(gb, orc):
    M = N = K = 8192
    vals, meta, dA, B, dB = _pruned(M, N, K, orc, 11)
    C = _sparse(gb, vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16)
    A_p = orc.decompress24(vals, meta, K)
    ms, ns = workloads.sample_pairs(M, N, 4096, seed=98)
    ms = np.concatenate([ms, np.repeat([0, M - 1], N), np.tile(np.arange(M), 2)])
    ns = np.concatenate([ns, np.tile(np.arange(N), 2), np.repeat([0, N - 1], M)])
    ref = orc.gemm_sampled(A_p, B, dA, 1, dB, 1, 1.0, ms, ns)
    S = orc.gemm_sampled(parity.abs_codes(A_p), parity.abs_codes(B), dA, 1, dB, 1, 1.0, ms, ns)
    parity.check_bf16(C[ms, ns], ref, S, K)


def test_gpu_prune_then_sparse_equals_dense_on_pruned(gb, orc):
    """GPU pipeline: prune on the device, sparse GEMM vs dense GEMM of the
    device-decompressed matrix (same operands, different kernels)."""
    M = N = K = 1024
    x = workloads.randn_f32((M, K), seed=41)
    w = workloads.randn_f32((N, K), seed=42)
    A, dA = gb.fp8_quantize_e4m3(_cuda(x), 1)
    B, dB = gb.fp8_quantize_e4m3(_cuda(w), 1)
    vals, meta = gb.prune24_compress(A)
    Ap = gb.prune24_decompress(vals, meta, K)
    Cs = gb.gemm_fp8_sparse24(vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_F32).double().cpu().numpy()
    Cd = gb.gemm_fp8_dense(Ap, B, dA, 1, dB, 1, 1.0, gb.OUT_F32).double().cpu().numpy()
    parity.check_fp32(Cs, Cd)


def test_k_not_multiple_of_128_rejected(gb):
    v = torch.zeros((4, 32), dtype=torch.uint8, device="cuda")
    m = torch.zeros((4, 8), dtype=torch.uint8, device="cuda")
    B = torch.zeros((4, 64), dtype=torch.uint8, device="cuda")
    s = torch.ones(1, device="cuda")
    with pytest.raises(gb.Fp8Error) as e:
        gb.gemm_fp8_sparse24(v, m, B, s, 0, s, 0)
    assert e.value.status == -2


def test_grouped_mixed_equals_single_bitwise(gb, orc):
    shapes = [(512, 768, 1024, True), (16, 2048, 512, False), (300, 200, 256, True),
              (1024, 256, 1024, False)]
    probs, outs, singles, keep = [], [], [], []
    for i, (M, N, K, sp) in enumerate(shapes):
        vals, meta, dA, B, dB = _pruned(M, N, K, orc, 30 + i)
        tB, tdA, tdB = _cuda(B), _cuda(dA), _cuda(dB)
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        if sp:
            tv, tm = _cuda(vals), _cuda(meta)
            keep += [tv, tm]
            probs.append(gb.make_problem(tv, tB, tdA, 1, tdB, 1, C, 1.0, gb.OUT_BF16, A_meta=tm))
            singles.append(gb.gemm_fp8_sparse24(tv, tm, tB, tdA, 1, tdB, 1, 1.0, gb.OUT_BF16))
        else:
            tA = _cuda(orc.decompress24(vals, meta, K))
            keep.append(tA)
            probs.append(gb.make_problem(tA, tB, tdA, 1, tdB, 1, C, 1.0, gb.OUT_BF16))
            singles.append(gb.gemm_fp8_dense(tA, tB, tdA, 1, tdB, 1, 1.0, gb.OUT_BF16))
        keep += [tB, tdA, tdB]
        outs.append(C)
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    for i, (C, Cs) in enumerate(zip(outs, singles)):
        assert torch.equal(C, Cs), i


@pytest.fixture()
def tile_cfg(gb):
    yield gb.fp8_gemm_set_tile_config
    gb.fp8_gemm_set_tile_config(0, 0)


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (300, 520, 768), (1000, 1500, 1024),
                                   (600, 17, 4096)])
def test_sparse_tile_configs_bitwise_equal_and_correct(gb, orc, tile_cfg, M, N, K):
    vals, meta, dA, B, dB = _pruned(M, N, K, orc, M + 3)
    outs = []
    for mt in (1, 2):
        tile_cfg(mt, 0)
        outs.append(_sparse(gb, vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_F32))
    assert np.array_equal(outs[0], outs[1])
    parity.check_fp32(outs[1], orc.gemm_sparse24(vals, meta, B, K, dA, 1, dB, 1))


def test_sparse_small_integers_mt2_bit_exact(gb, orc, tile_cfg):
    A = workloads.small_int_codes((384, 1024), seed=77)
    B = workloads.small_int_codes((300, 1024), seed=78)
    vals, meta = orc.prune24(A)
    one = np.ones(1, np.float32)
    tile_cfg(2, 0)
    C = _sparse(gb, vals, meta, B, one, 0, one, 0, 1.0, gb.OUT_F32)
    assert np.array_equal(C.astype(np.float64), orc.gemm_sparse24(vals, meta, B, 1024, one, 0, one, 0))


@pytest.mark.parametrize("M,N,K", [(256, 128, 262144), (128, 16, 131072), (1 << 19, 16, 128)])
def test_sparse_extreme_shapes_small_integers_exact(gb, orc, M, N, K):
    """2:4 products at very long K and at half a million rows: every entry
    equals the integer product of the pruned matrix with B, sampled entries
    equal the oracle's."""
    A = workloads.small_int_codes((M, K), seed=M + 21)
    B = workloads.small_int_codes((N, K), seed=N + 22)
    vals, meta = orc.prune24(A)
    one = np.ones(1, np.float32)
    C = _sparse(gb, vals, meta, B, one, 0, one, 0, 1.0, gb.OUT_F32)
    Ap = orc.decompress24(vals, meta, K)
    exact = torch.from_numpy(Ap).view(torch.float8_e4m3fn).double().numpy() @ \
        workloads.randint_f32((N, K), N + 22, -4, 4).astype(np.float64).T
    assert np.array_equal(C.astype(np.float64), exact)
    ms, ns = workloads.sample_pairs(M, N, 256, seed=10)
    assert np.array_equal(C[ms, ns].astype(np.float64), orc.gemm_sampled(Ap, B, one, 0, one, 0, 1.0, ms, ns))
