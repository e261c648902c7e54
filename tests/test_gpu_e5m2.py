"""GPU parity for the second FP8 operand format, E5M2 ("bf8", paper section
2), and for mixed E4M3 x E5M2 operands (the four pairings of paper Table 3):
fp8_quantize_e5m2 bit-exact against the oracle; gemm_fp8_dense_fmt,
gemm_fp8_sparse24_fmt and grouped problems with per-operand formats against
the FP64 oracle (bit-exact on small-integer codes, tolerances of
tests/parity.py otherwise), on every launch path: 128- and 256-row tiles,
the swapped skinny path (the formats travel with their operands), split-K
through the workspace and through a cluster, and ragged edges."""
import numpy as np
import pytest
import torch

import workloads
from tests import parity

pytestmark = pytest.mark.gpu

PAIRS = [(0, 0), (0, 1), (1, 0), (1, 1)]


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _codes(a):
    """Device copy with the row stride padded to a multiple of 16 bytes."""
    M, K = a.shape
    ld = max(16, (K + 15) // 16 * 16)
    t = torch.zeros((M, ld), dtype=torch.uint8, device="cuda")
    t[:, :K] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t[:, :K]


def _ok(gb):
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0


# --- quantisation ----------------------------------------------------------------

def _quant(gb, x, mode):
    q, d = gb.fp8_quantize_e5m2(torch.from_numpy(x).cuda(), mode)
    _ok(gb)
    return q.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (33, 3), (257, 1000), (64, 4096), (1000, 1029)])
def test_quantize_parity(gb, orc, mode, shape):
    x = workloads.randn_f32(shape, seed=shape[0] * 7 + shape[1])
    q, d = _quant(gb, x, mode)
    qo, do = orc.quantize(x, mode, fmt=1)
    assert np.array_equal(q, qo)
    assert np.array_equal(d, do)


@pytest.mark.parametrize("mode", [0, 1])
def test_quantize_parity_full_size(gb, orc, mode):
    # the square-sweep operand size (8192 x 8192 fp32)
    x = workloads.randn_f32((8192, 8192), seed=41 + mode)
    q, d = _quant(gb, x, mode)
    qo, do = orc.quantize(x, mode, fmt=1)
    assert np.array_equal(q, qo)
    assert np.array_equal(d, do)


def test_quantize_wide_dynamic_range(gb, orc):
    # rows spanning many binades: tiny values land in E5M2's subnormals
    x = workloads.randn_f32((64, 2048), seed=43)
    x *= np.float32(2.0) ** workloads.randint_f32((64, 2048), 44, -30, 10)
    for mode in (0, 1):
        q, d = _quant(gb, x, mode)
        qo, do = orc.quantize(x, mode, fmt=1)
        assert np.array_equal(q, qo) and np.array_equal(d, do)
        assert np.count_nonzero((q & 0x7F) < 4) > 0          # subnormals and zeros occur


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("mode", [0, 1])
def test_quantize_nonfinite_reported(gb, mode, bad):
    x = np.ones((8, 64), np.float32)
    x[5, 3] = bad
    gb.fp8_quantize_e5m2(torch.from_numpy(x).cuda(), mode)
    assert gb.fp8_last_device_error() == -4
    assert gb.fp8_last_device_error() == 0


def test_device_encoder_all_in_range_fp32(gb, orc):
    """Every fp32 bit pattern with |x| <= 57344 through the device encoder:
    a tensor whose amax is exactly 57344 gets s = 1, so the codes are enc(x)."""
    top = 0x47600000                                     # bits of 57344.0f
    chunk = 1 << 26
    cols = 1024
    for sign in (0, 0x80000000):
        for lo in range(0, top + 1, chunk):
            hi = min(lo + chunk, top + 1)
            n = hi - lo
            rows = (n + cols - 1) // cols
            bits = torch.arange(lo, lo + rows * cols, dtype=torch.int64, device="cuda")
            bits = torch.clamp(bits, max=hi - 1) | sign
            bits = torch.where(bits >= 2 ** 31, bits - 2 ** 32, bits)
            x = bits.to(torch.int32).view(torch.float32).reshape(rows, cols)
            x = torch.cat([x, torch.full((1, cols), 57344.0, device="cuda")])
            q, d = gb.fp8_quantize_e5m2(x, 0)
            assert d.item() == 1.0
            got = q[:-1].reshape(-1)[:n].cpu().numpy()
            ref = orc.e5m2_encode_pattern_range(lo | sign, (hi - 1 | sign) + 1)
            assert np.array_equal(got, ref), f"chunk at {lo | sign:#x}"


# --- dense GEMM with per-operand formats -------------------------------------------

def _dense(gb, A, B, dA, a_mode, dB, b_mode, alpha, out_dtype, af, bf):
    C = gb.gemm_fp8_dense_fmt(_codes(A), _codes(B), _cuda(dA), a_mode, _cuda(dB), b_mode, alpha,
                              out_dtype, af, bf)
    _ok(gb)
    return C.float().cpu().numpy()


def _quantized(M, N, K, orc, af, bf, seed):
    x = workloads.randn_f32((M, K), seed=workloads.SEED_A + seed)
    w = workloads.randn_f32((N, K), seed=workloads.SEED_B + seed)
    A, dA = orc.quantize(x, 1, fmt=af)
    B, dB = orc.quantize(w, 1, fmt=bf)
    return A, dA, B, dB


@pytest.mark.parametrize("af,bf", PAIRS)
@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (200, 72, 320), (16, 512, 1024), (1, 1, 1),
                                   (300, 17, 4100), (513, 700, 1000)])
def test_dense_small_integers_bit_exact(gb, orc, af, bf, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + 3, maxabs=8, fmt=af)
    B = workloads.small_int_codes((N, K), seed=N + 4, maxabs=8, fmt=bf)
    one = np.ones(1, np.float32)
    C = _dense(gb, A, B, one, 0, one, 0, 1.0, gb.OUT_F32, af, bf)
    assert np.array_equal(C.astype(np.float64), orc.gemm(A, B, one, 0, one, 0, a_fmt=af, b_fmt=bf))


@pytest.mark.parametrize("af,bf", PAIRS)
@pytest.mark.parametrize("M,N,K", [(1024, 1024, 1024), (1000, 1500, 700), (16, 8192, 1024),
                                   (64, 3000, 512), (129, 333, 256)])
def test_dense_bf16_per_row(gb, orc, af, bf, M, N, K):
    A, dA, B, dB = _quantized(M, N, K, orc, af, bf, seed=M + 10 * af + 20 * bf)
    C = _dense(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, af, bf)
    ref = orc.gemm(A, B, dA, 1, dB, 1, a_fmt=af, b_fmt=bf)
    S = orc.gemm(parity.abs_codes(A), parity.abs_codes(B), dA, 1, dB, 1, a_fmt=af, b_fmt=bf)
    parity.check_bf16(C, ref, S, K)


@pytest.mark.parametrize("af,bf", PAIRS)
def test_dense_random_codes_fp32(gb, orc, af, bf):
    # every finite code of each format, values from 2^-16 (or 2^-9) to 57344
    M, N, K = 300, 260, 640
    A = workloads.random_codes((M, K), seed=50 + af, fmt=af)
    B = workloads.random_codes((N, K), seed=60 + bf, fmt=bf)
    dA = np.abs(workloads.randn_f32((M,), seed=3)) + 0.5
    dB = np.abs(workloads.randn_f32((N,), seed=4)) + 0.5
    C = _dense(gb, A, B, dA, 1, dB, 1, -0.75, gb.OUT_F32, af, bf)
    parity.check_fp32(C, orc.gemm(A, B, dA, 1, dB, 1, -0.75, a_fmt=af, b_fmt=bf))


@pytest.mark.parametrize("af,bf", [(0, 1), (1, 0)])
@pytest.mark.parametrize("M,N,K", [(16, 4096, 4096), (16, 8192, 8192), (40, 2048, 8192),
                                   (1, 2048, 4096)])
def test_dense_split_k_paths(gb, orc, af, bf, M, N, K):
    """Skinny products: A goes to the MMA N side (its format with it) and K is
    split through the workspace or a cluster."""
    A, dA, B, dB = _quantized(M, N, K, orc, af, bf, seed=M + K)
    C = _dense(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_F32, af, bf)
    parity.check_fp32(C, orc.gemm(A, B, dA, 1, dB, 1, a_fmt=af, b_fmt=bf))


def test_format_is_not_ignored(gb, orc):
    # the same bytes under the four pairings give four different products,
    # each equal to the oracle's
    M, N, K = 128, 128, 256
    A = workloads.small_int_codes((M, K), seed=70, maxabs=4, fmt=0)
    B = workloads.small_int_codes((N, K), seed=71, maxabs=4, fmt=0)
    one = np.ones(1, np.float32)
    outs = []
    for af, bf in PAIRS:
        C = _dense(gb, A, B, one, 0, one, 0, 1.0, gb.OUT_F32, af, bf)
        ref = orc.gemm(A, B, one, 0, one, 0, a_fmt=af, b_fmt=bf)
        parity.check_fp32(C, ref)
        outs.append(C)
    for i in range(4):
        for j in range(i):
            assert not np.array_equal(outs[i], outs[j])


def test_e4m3_pair_equals_plain_entry_point(gb, orc):
    A, dA, B, dB = _quantized(384, 500, 1024, orc, 0, 0, seed=80)
    C1 = gb.gemm_fp8_dense(_codes(A), _codes(B), _cuda(dA), 1, _cuda(dB), 1, 1.0, gb.OUT_BF16)
    C2 = gb.gemm_fp8_dense_fmt(_codes(A), _codes(B), _cuda(dA), 1, _cuda(dB), 1, 1.0, gb.OUT_BF16,
                               gb.E4M3, gb.E4M3)
    _ok(gb)
    assert torch.equal(C1, C2)


@pytest.mark.parametrize("af,bf", [(1, 1), (0, 1)])
def test_dense_full_size_sampled(gb, orc, af, bf):
    M = N = K = 8192
    A, dA, B, dB = _quantized(M, N, K, orc, af, bf, seed=90 + af)
    C = _dense(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, af, bf)
    ms, ns = workloads.sample_pairs(M, N, 4096, seed=98)
    ref = orc.gemm_sampled(A, B, dA, 1, dB, 1, 1.0, ms, ns, a_fmt=af, b_fmt=bf)
    S = orc.gemm_sampled(parity.abs_codes(A), parity.abs_codes(B), dA, 1, dB, 1, 1.0, ms, ns,
                         a_fmt=af, b_fmt=bf)
    parity.check_bf16(C[ms, ns], ref, S, K)


# --- 2:4 sparse and grouped ----------------------------------------------------------

@pytest.mark.parametrize("af,bf", PAIRS)
@pytest.mark.parametrize("M,N,K", [(128, 128, 128), (200, 72, 384), (16, 512, 1024),
                                   (300, 17, 4096)])
def test_sparse_small_integers_bit_exact(gb, orc, af, bf, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + 5, maxabs=8, fmt=af)
    B = workloads.small_int_codes((N, K), seed=N + 6, maxabs=8, fmt=bf)
    vals, meta = orc.prune24(A)
    one = np.ones(1, np.float32)
    C = gb.gemm_fp8_sparse24_fmt(_cuda(vals), _cuda(meta), _cuda(B), _cuda(one), 0, _cuda(one), 0,
                                 1.0, gb.OUT_F32, False, af, bf)
    _ok(gb)
    ref = orc.gemm_sparse24(vals, meta, B, K, one, 0, one, 0, a_fmt=af, b_fmt=bf)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("af,bf", [(1, 0), (1, 1)])
def test_sparse_device_prune_bf16_transposed(gb, orc, af, bf):
    M, N, K = 1000, 700, 1024
    A, dA, B, dB = _quantized(M, N, K, orc, af, bf, seed=110 + bf)
    vals_d, meta_d = gb.prune24_compress(_cuda(A))
    vals, meta = orc.prune24(A)
    assert np.array_equal(vals_d.cpu().numpy(), vals)
    assert np.array_equal(meta_d.cpu().numpy(), meta)
    C = gb.gemm_fp8_sparse24_fmt(vals_d, meta_d, _cuda(B), _cuda(dA), 1, _cuda(dB), 1, 0.5,
                                 gb.OUT_BF16, True, af, bf)
    _ok(gb)
    ref = orc.gemm_sparse24(vals, meta, B, K, dA, 1, dB, 1, 0.5, a_fmt=af, b_fmt=bf)
    S = orc.gemm_sparse24(parity.abs_codes(vals), meta, parity.abs_codes(B), K, dA, 1, dB, 1, 0.5,
                          a_fmt=af, b_fmt=bf)
    parity.check_bf16(C.float().cpu().numpy().T, ref, S, K)


def test_grouped_mixed_formats_equal_single_calls(gb, orc):
    """One persistent launch holding problems of all four pairings (dense and
    sparse): each equals its own single call bit for bit."""
    shapes = [(512, 768, 1024, 0, 1), (16, 2048, 512, 1, 0), (300, 200, 256, 1, 1),
              (256, 384, 2048, 0, 0), (384, 256, 1024, 1, 0)]
    probs, outs, singles, keep = [], [], [], []
    for i, (M, N, K, af, bf) in enumerate(shapes):
        A, dA, B, dB = _quantized(M, N, K, orc, af, bf, seed=120 + i)
        t = [_cuda(A), _cuda(B), _cuda(dA), _cuda(dB)]
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        if i == 4:                                       # a sparse problem
            vals, meta = gb.prune24_compress(t[0])
            t += [vals, meta]
            probs.append(gb.make_problem(vals, t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16,
                                         A_meta=meta, a_format=af, b_format=bf))
            singles.append(gb.gemm_fp8_sparse24_fmt(vals, meta, t[1], t[2], 1, t[3], 1, 1.0,
                                                    gb.OUT_BF16, False, af, bf))
        else:
            probs.append(gb.make_problem(t[0], t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16,
                                         a_format=af, b_format=bf))
            singles.append(gb.gemm_fp8_dense_fmt(t[0], t[1], t[2], 1, t[3], 1, 1.0, gb.OUT_BF16,
                                                 af, bf))
        keep += t
        outs.append(C)
    gb.gemm_fp8_grouped(probs)
    _ok(gb)
    for C, Cs in zip(outs, singles):
        assert torch.equal(C, Cs)
