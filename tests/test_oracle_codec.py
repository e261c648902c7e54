"""Pins for the oracle's E4M3 codec (OCP E4M3, paper section 2).

The oracle is checked against things other than itself: PyTorch's and
ml_dtypes' float8_e4m3fn conversions (library routines), the OCP table of
landmark values, and a brute-force nearest-value encoder over every fp32 bit
pattern of one sign plus a sampled other sign.
"""
import os

import numpy as np
import pytest
import torch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _torch_decode_all():
    codes = torch.arange(256, dtype=torch.int32).to(torch.uint8)
    return codes.view(torch.float8_e4m3fn).to(torch.float64).numpy()


def test_decode_all_256_codes_vs_torch(orc):
    ours = orc.e4m3_decode(np.arange(256, dtype=np.uint8))
    ref = _torch_decode_all()
    nan = np.isnan(ref)
    assert list(np.nonzero(nan)[0]) == [0x7F, 0xFF]
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])
    # the sign of zero is part of the code
    assert np.signbit(ours[0x80]) and not np.signbit(ours[0x00])


def test_decode_all_256_codes_vs_ml_dtypes(orc):
    ml_dtypes = pytest.importorskip("ml_dtypes")
    ref = np.arange(256, dtype=np.uint8).view(ml_dtypes.float8_e4m3fn).astype(np.float64)
    ours = orc.e4m3_decode(np.arange(256, dtype=np.uint8))
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])


def _landmarks():
    rows = []
    with open(os.path.join(GOLDEN, "e4m3_landmarks.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                c, v = line.split()
                rows.append((int(c, 16), float(v)))
    return rows


def test_decode_landmarks(orc):
    rows = _landmarks()
    assert len(rows) >= 10
    for code, val in rows:
        got = orc.e4m3_decode(np.array([code], np.uint8))[0]
        if np.isnan(val):
            assert np.isnan(got), hex(code)
        else:
            assert got == val and np.signbit(got) == np.signbit(val), hex(code)


def test_encode_landmarks_roundtrip(orc):
    for code, val in _landmarks():
        if not np.isnan(val):
            assert int(orc.e4m3_encode(np.float32(val))) == code, hex(code)


def _all_midpoints():
    """Every midpoint between adjacent finite positive codes, and the fp32
    neighbours on each side of it."""
    vals = _torch_decode_all()[:0x7F]
    mids = (vals[:-1] + vals[1:]) / 2.0
    m32 = mids.astype(np.float32)
    assert np.array_equal(m32.astype(np.float64), mids)     # exact in fp32
    up = np.nextafter(m32, np.float32(np.inf))
    dn = np.nextafter(m32, np.float32(0))
    return np.concatenate([m32, up, dn])


def test_encode_vs_torch_in_range(orc):
    # torch's cast is round-to-nearest-even without saturation; it agrees with
    # the oracle wherever the rounded result is finite (|x| < 464).
    rng = np.random.default_rng(0)
    x = np.concatenate([
        _all_midpoints(),
        rng.standard_normal(200000).astype(np.float32) * np.float32(60.0),
        (rng.random(200000).astype(np.float32) * np.float32(2 ** -5)),
        np.array([0.0, 2 ** -10, 2 ** -11, 3 * 2 ** -10, 447.9, 463.9], np.float32),
    ])
    x = np.concatenate([x, -x])
    ours = orc.e4m3_encode(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)


def test_encode_saturates(orc):
    big = np.array([448.0, 464.0, 500.0, 1e6, 3.0e38, np.inf], np.float32)
    assert np.all(orc.e4m3_encode(big) == 0x7E)
    assert np.all(orc.e4m3_encode(-big) == 0xFE)
    nan = orc.e4m3_encode(np.array([np.nan], np.float32))[0]
    assert nan & 0x7F == 0x7F


def test_encode_linear_scan_equals_search(orc):
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    xs = np.concatenate([bits.view(np.float32), _all_midpoints()])
    for x in xs:
        assert orc.e4m3_encode_bruteforce(float(x)) == orc.e4m3_encode_search(float(x)), x


@pytest.mark.slow
def test_encode_exhaustive_positive_fp32(orc):
    # every fp32 bit pattern with the sign bit clear (2^31 patterns)
    bad, first = orc.check_encoder_range(0, 1 << 31)
    assert bad == 0, hex(first)


@pytest.mark.slow
def test_encode_exhaustive_negative_fp32(orc):
    # and every pattern with the sign bit set: with the positive half, all 2^32
    bad, first = orc.check_encoder_range(1 << 31, 1 << 32)
    assert bad == 0, hex(first)


def test_encode_sampled_negative_fp32(orc):
    # the negative half on a fixed stride plus the symmetry encode(-x) = encode(x) ^ 0x80
    lo = 1 << 31
    for start in range(lo, 1 << 32, 1 << 27):
        bad, first = orc.check_encoder_range(start, start + (1 << 16))
        assert bad == 0, hex(first)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(100000).astype(np.float32) * np.float32(100)
    assert np.array_equal(orc.e4m3_encode(-x), orc.e4m3_encode(x) ^ 0x80)
