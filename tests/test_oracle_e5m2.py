"""Pins for the oracle's E5M2 codec, E5M2 quantisation and mixed-format GEMM
(OCP E5M2, the "bf8" operand type of paper section 2; the four FP8/BF8
operand pairings of Table 3).

Checked against things other than the oracle itself: PyTorch's and
ml_dtypes' float8_e5m2 conversions (library routines), the OCP table of
landmark values, the IEEE binary16 layout (an E5M2 code is the high byte of
the binary16 encoding of the same value; rounding a binary16 pattern to its
high byte with the integer round-half-even rule gives the E5M2 code of every
binary16 value), a brute-force nearest-value scan, and numpy float64 matmul
on operands decoded by PyTorch.
"""
import os

import numpy as np
import pytest
import torch

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MAXF = 57344.0


def _torch_decode_all():
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    return codes.view(torch.float8_e5m2).to(torch.float64).numpy()


def _torch_decode(codes, fmt):
    dt = torch.float8_e5m2 if fmt == 1 else torch.float8_e4m3fn
    return torch.from_numpy(np.ascontiguousarray(codes)).view(dt).to(torch.float64).numpy()


# --- decode -------------------------------------------------------------------

def test_decode_all_256_codes_vs_torch(orc):
    ours = orc.e5m2_decode(np.arange(256, dtype=np.uint8))
    ref = _torch_decode_all()
    nan = np.isnan(ref)
    assert list(np.nonzero(nan)[0]) == [0x7D, 0x7E, 0x7F, 0xFD, 0xFE, 0xFF]
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])
    assert ours[0x7C] == np.inf and ours[0xFC] == -np.inf
    assert np.signbit(ours[0x80]) and not np.signbit(ours[0x00])


def test_decode_all_256_codes_vs_ml_dtypes(orc):
    ml_dtypes = pytest.importorskip("ml_dtypes")
    ref = np.arange(256, dtype=np.uint8).view(ml_dtypes.float8_e5m2).astype(np.float64)
    ours = orc.e5m2_decode(np.arange(256, dtype=np.uint8))
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])


def test_decode_is_high_byte_of_binary16(orc):
    # code c has the value of the binary16 pattern c << 8 (numpy's float16)
    h = (np.arange(256, dtype=np.uint16) << 8).view(np.float16).astype(np.float64)
    ours = orc.e5m2_decode(np.arange(256, dtype=np.uint8))
    nan = np.isnan(h)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], h[~nan])


def _landmarks():
    rows = []
    with open(os.path.join(GOLDEN, "e5m2_landmarks.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                c, v = line.split()
                rows.append((int(c, 16), float(v)))
    return rows


def test_decode_landmarks(orc):
    rows = _landmarks()
    assert len(rows) >= 15
    for code, val in rows:
        got = orc.e5m2_decode(np.array([code], np.uint8))[0]
        if np.isnan(val):
            assert np.isnan(got), hex(code)
        else:
            assert got == val and np.signbit(got) == np.signbit(val), hex(code)


def test_encode_landmarks_roundtrip(orc):
    for code, val in _landmarks():
        if np.isfinite(val):
            assert int(orc.e5m2_encode(np.float32(val))) == code, hex(code)


# --- encode -------------------------------------------------------------------

def _all_midpoints():
    """Every midpoint between adjacent finite positive codes and the fp32
    neighbours on each side of it."""
    vals = _torch_decode_all()[:0x7C]
    mids = (vals[:-1] + vals[1:]) / 2.0
    m32 = mids.astype(np.float32)
    assert np.array_equal(m32.astype(np.float64), mids)     # exact in fp32
    up = np.nextafter(m32, np.float32(np.inf))
    dn = np.nextafter(m32, np.float32(0))
    return np.concatenate([m32, up, dn])


def test_encode_vs_torch_in_range(orc):
    # torch's cast rounds to nearest even without saturation; it agrees with
    # the oracle wherever the rounded result is finite (|x| < 61440).
    rng = np.random.default_rng(10)
    x = np.concatenate([
        _all_midpoints(),
        rng.standard_normal(200000).astype(np.float32) * np.float32(8000.0),
        rng.random(200000).astype(np.float32) * np.float32(2 ** -12),
        np.array([0.0, 2 ** -17, 3 * 2 ** -18, 2 ** -18, 57343.0, 61439.0, 1e-30], np.float32),
    ])
    x = np.concatenate([x, -x])
    ours = orc.e5m2_encode(x)
    ref = torch.from_numpy(x).to(torch.float8_e5m2).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)


def test_encode_every_binary16_by_integer_rounding(orc):
    # For a binary16 value with pattern h, the nearest E5M2 code (ties to even)
    # is h / 256 rounded half-to-even as an integer: E5M2 keeps the top byte
    # and both formats space their codes uniformly within a binade, with the
    # same subnormal step structure.  Finite binary16 below the overflow
    # threshold 61440 (pattern 0x7B80) only.
    h = np.arange(0x7B80, dtype=np.uint32)
    low = h & 0xFF
    hi = h >> 8
    up = (low > 0x80) | ((low == 0x80) & ((hi & 1) == 1))
    ref = (hi + up).astype(np.uint8)
    x = h.astype(np.uint16).view(np.float16).astype(np.float32)
    assert np.array_equal(orc.e5m2_encode(x), ref)
    assert np.array_equal(orc.e5m2_encode(-x), ref | 0x80)


def test_encode_saturates(orc):
    big = np.array([MAXF, 60000.0, 61440.0, 65504.0, 1e6, 3.0e38, np.inf], np.float32)
    assert np.all(orc.e5m2_encode(big) == 0x7B)
    assert np.all(orc.e5m2_encode(-big) == 0xFB)
    nan = orc.e5m2_encode(np.array([np.nan, -np.nan], np.float32))
    assert np.all(nan & 0x7F == 0x7F)


def test_encode_linear_scan_equals_search(orc):
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    xs = np.concatenate([bits.view(np.float32), _all_midpoints(), -_all_midpoints()])
    for x in xs:
        assert orc.e5m2_encode_bruteforce(float(x)) == orc.e5m2_encode_search(float(x)), x


@pytest.mark.slow
def test_encode_exhaustive_positive_fp32(orc):
    bad, first = orc.check_e5m2_encoder_range(0, 1 << 31)
    assert bad == 0, hex(first)


@pytest.mark.slow
def test_encode_exhaustive_negative_fp32(orc):
    bad, first = orc.check_e5m2_encoder_range(1 << 31, 1 << 32)
    assert bad == 0, hex(first)


def test_encode_sampled_negative_fp32(orc):
    lo = 1 << 31
    for start in range(lo, 1 << 32, 1 << 27):
        bad, first = orc.check_e5m2_encoder_range(start, start + (1 << 16))
        assert bad == 0, hex(first)
    rng = np.random.default_rng(12)
    x = rng.standard_normal(100000).astype(np.float32) * np.float32(1e4)
    assert np.array_equal(orc.e5m2_encode(-x), orc.e5m2_encode(x) ^ 0x80)


def test_pattern_range_equals_array_encoder(orc):
    lo = 0x47000000                               # 32768.0f
    got = orc.e5m2_encode_pattern_range(lo, lo + 4096)
    x = np.arange(lo, lo + 4096, dtype=np.uint32).view(np.float32)
    assert np.array_equal(got, orc.e5m2_encode(x))


# --- quantisation -------------------------------------------------------------

def test_quantize_closed_form(orc):
    # amax 7 per row 0 -> s = fl32(57344 / 7) = 8192 exactly, d = 7 / 57344;
    # 7 * 8192 = 57344 = S.11110.11 (0x7B), 3.5 * 8192 = 1.75 * 2^14 =
    # S.11101.11 (0x77), 1 * 8192 = 2^13 = S.11100.00 (0x70),
    # -2 * 8192 = -2^14 = S.11101.00 with the sign bit (0xF4).
    x = np.array([[7.0, 3.5, 1.0, -2.0], [0.0, 0.0, 0.0, 0.0]], np.float32)
    q, d = orc.quantize(x, 1, fmt=1)
    assert list(q[0]) == [0x7B, 0x77, 0x70, 0xF4]
    assert list(q[1]) == [0, 0, 0, 0]
    assert d[0] == np.float32(7.0) / np.float32(MAXF) and d[1] == 1.0


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape", [(3, 17), (64, 256)])
def test_quantize_matches_torch_restatement(orc, mode, shape):
    x = workloads.randn_f32(shape, seed=77 + mode)
    q, d = orc.quantize(x, mode, fmt=1)
    xt = torch.from_numpy(x)
    amax = xt.abs().amax(dim=1, keepdim=True) if mode else xt.abs().amax().reshape(1, 1)
    s = torch.tensor(MAXF, dtype=torch.float32) / amax
    ref = (xt * s).to(torch.float8_e5m2).view(torch.uint8).numpy()
    assert np.array_equal(q, ref)
    assert np.array_equal(d, (amax / torch.tensor(MAXF)).reshape(-1).numpy())


def test_quantize_amax_maps_to_max(orc):
    x = workloads.randn_f32((16, 300), seed=5)
    q, _ = orc.quantize(x, 1, fmt=1)
    i = np.argmax(np.abs(x), axis=1)
    top = q[np.arange(16), i]
    assert np.all(top & 0x7F == 0x7B)
    assert np.all((top >> 7) == (x[np.arange(16), i] < 0))
    assert np.all(q & 0x7F <= 0x7B)                   # never inf or NaN


def test_quantize_formats_differ_only_in_target(orc):
    # the same scaled product, encoded by two formats: E4M3 quantisation with
    # amax mapped to 448 and E5M2 with amax mapped to 57344 = 128 * 448 give
    # values whose ratio is 128 up to each format's rounding (<= 2^-4 and
    # 2^-3 relative for normals)
    x = workloads.randn_f32((8, 512), seed=6)
    q4, d4 = orc.quantize(x, 1, fmt=0)
    q5, d5 = orc.quantize(x, 1, fmt=1)
    v4 = orc.e4m3_decode(q4) * d4[:, None]
    v5 = orc.e5m2_decode(q5) * d5[:, None]
    big = np.abs(x) > 0.1
    assert np.all(np.abs(v4 - x)[big] <= 2 ** -4 * np.abs(x)[big] * 1.001)
    assert np.all(np.abs(v5 - x)[big] <= 2 ** -3 * np.abs(x)[big] * 1.001)
    assert np.allclose(d5 * 128, d4, rtol=2 ** -22)


def test_quantize_rejects_bad_format(orc):
    import oracle
    with pytest.raises(oracle.OracleError):
        orc.quantize(np.ones((2, 2), np.float32), 0, fmt=2)


# --- GEMM with per-operand formats -----------------------------------------------

@pytest.mark.parametrize("a_fmt,b_fmt", [(0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K,a_mode,b_mode", [(17, 9, 64, 1, 1), (3, 5, 7, 0, 0)])
def test_gemm_formats_vs_numpy(orc, a_fmt, b_fmt, M, N, K, a_mode, b_mode):
    A = workloads.random_codes((M, K), seed=M, fmt=a_fmt)
    B = workloads.random_codes((N, K), seed=N + 100, fmt=b_fmt)
    dA = np.abs(workloads.randn_f32((M,), seed=3)) + 0.5
    dB = np.abs(workloads.randn_f32((N,), seed=4)) + 0.5
    C = orc.gemm(A, B, dA, a_mode, dB, b_mode, 0.75, a_fmt=a_fmt, b_fmt=b_fmt)
    sa = dA.astype(np.float64) if a_mode else np.full(M, float(dA[0]))
    sb = dB.astype(np.float64) if b_mode else np.full(N, float(dB[0]))
    ref = 0.75 * sa[:, None] * sb[None, :] * (_torch_decode(A, a_fmt) @ _torch_decode(B, b_fmt).T)
    np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-300)


def test_gemm_small_integers_exact_every_pairing(orc):
    M, N, K = 12, 10, 96
    for a_fmt in (0, 1):
        for b_fmt in (0, 1):
            A = workloads.small_int_codes((M, K), seed=21, maxabs=8, fmt=a_fmt)
            B = workloads.small_int_codes((N, K), seed=22, maxabs=8, fmt=b_fmt)
            ia = workloads.randint_f32((M, K), 21, -8, 8).astype(np.int64)
            ib = workloads.randint_f32((N, K), 22, -8, 8).astype(np.int64)
            C = orc.gemm(A, B, np.ones(1, np.float32), 0, np.ones(1, np.float32), 0, 1.0,
                         a_fmt=a_fmt, b_fmt=b_fmt)
            assert np.array_equal(C, (ia @ ib.T).astype(np.float64)), (a_fmt, b_fmt)


def test_gemm_format_is_per_operand(orc):
    # the same bytes read as E4M3 and as E5M2 give different products; the
    # format of one operand must not leak into the other
    A = workloads.random_codes((4, 32), seed=1)
    B = np.full((3, 32), 0x3C, np.uint8)                # E5M2 1.0 (E4M3 1.5)
    one = np.ones(1, np.float32)
    C = orc.gemm(A, B, one, 0, one, 0, 1.0, a_fmt=0, b_fmt=1)
    np.testing.assert_array_equal(C, np.repeat(orc.e4m3_decode(A).sum(1)[:, None], 3, 1))
    C2 = orc.gemm(A, B, one, 0, one, 0, 1.0, a_fmt=0, b_fmt=0)
    np.testing.assert_array_equal(C2, 1.5 * C)


def test_gemm_sampled_and_sparse_carry_formats(orc):
    M, N, K = 24, 16, 64
    A = workloads.random_codes((M, K), seed=7, fmt=1)
    B = workloads.random_codes((N, K), seed=8, fmt=0)
    dA = np.abs(workloads.randn_f32((M,), seed=9)) + 0.5
    dB = np.abs(workloads.randn_f32((N,), seed=10)) + 0.5
    full = orc.gemm(A, B, dA, 1, dB, 1, 1.25, a_fmt=1, b_fmt=0)
    ms, ns = workloads.sample_pairs(M, N, 50, seed=3)
    samp = orc.gemm_sampled(A, B, dA, 1, dB, 1, 1.25, ms, ns, a_fmt=1, b_fmt=0)
    np.testing.assert_array_equal(samp, full[ms, ns])
    vals, meta = orc.prune24(A)
    pruned = orc.decompress24(vals, meta, K)
    sp = orc.gemm_sparse24(vals, meta, B, K, dA, 1, dB, 1, 1.25, a_fmt=1, b_fmt=0)
    np.testing.assert_array_equal(sp, orc.gemm(pruned, B, dA, 1, dB, 1, 1.25, a_fmt=1, b_fmt=0))


def test_prune_keeps_largest_e5m2_magnitudes(orc):
    # the pruning key (code & 0x7F) orders finite E5M2 codes by magnitude too:
    # the kept pair of every group holds the two largest |values| (decoded by
    # torch), ties aside
    A = workloads.random_codes((32, 128), seed=12, fmt=1)
    vals, meta = orc.prune24(A)
    dec = np.abs(_torch_decode(A, 1)).reshape(32, 32, 4)
    kept = np.abs(_torch_decode(vals, 1)).reshape(32, 32, 2)
    top2 = -np.sort(-dec, axis=2)[:, :, :2]
    np.testing.assert_array_equal(np.sort(kept, axis=2), np.sort(top2, axis=2))
