"""Pins for the oracle's block-scaled FP8 (OCP MX: MXFP8 E4M3 / E5M2 with
E8M0 block scales; not in the paper, the next precision step after its
per-row scaling).

Checked against things other than the oracle itself: PyTorch's and
ml_dtypes' float8_e8m0fnu decode, hand-worked blocks, the defining property
of the scale (the block maximum lands in the element format's top binade)
checked in float64, PyTorch's FP8 casts of the scaled block, power-of-two
invariance, and numpy float64 matmul on operands decoded by PyTorch.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

EMAX = {0: 8, 1: 15}
MAXF = {0: 448.0, 1: 57344.0}
TORCH_FP8 = {0: torch.float8_e4m3fn, 1: torch.float8_e5m2}


def _dec(codes, fmt):
    return torch.from_numpy(np.ascontiguousarray(codes)).view(TORCH_FP8[fmt]).to(torch.float64).numpy()


def test_e8m0_decode_all_codes_vs_torch_and_ml_dtypes(orc):
    c = np.arange(256, dtype=np.uint8)
    ours = orc.e8m0_decode(c)
    ref = torch.from_numpy(c).view(torch.float8_e8m0fnu).to(torch.float64).numpy()
    assert np.isnan(ours[255]) and np.isnan(ref[255])
    assert np.array_equal(ours[:255], ref[:255])
    assert ours[127] == 1.0 and ours[0] == 2.0 ** -127 and ours[254] == 2.0 ** 127
    ml_dtypes = pytest.importorskip("ml_dtypes")
    ref2 = c.view(ml_dtypes.float8_e8m0fnu).astype(np.float64)
    assert np.array_equal(ours[:255], ref2[:255])


def test_hand_worked_blocks(orc):
    # E4M3, block {1, 0.5, 0...}: amax 1 = 2^0 -> e = 0 - 8 = -8 (code 119);
    # 1 * 2^8 = 256 = S.1111.000 (0x78), 0.5 * 2^8 = 128 = S.1110.000 (0x70).
    # Block {-3, 1, 0.5, 0...}: amax 3, floor(log2 3) = 1 -> e = -7 (code 120);
    # -3 * 2^7 = -384 = -1.5 * 2^8 (0xFC), 1 * 2^7 = 128 (0x70), 0.5 * 2^7 =
    # 64 = S.1101.000 (0x68).
    x = np.zeros((2, 32), np.float32)
    x[0, 0], x[0, 1] = 1.0, 0.5
    x[1, 0], x[1, 1], x[1, 2] = -3.0, 1.0, 0.5
    q, s = orc.mx_quantize(x, 0)
    assert s.tolist() == [[119], [120]]
    assert q[0, :2].tolist() == [0x78, 0x70] and not q[0, 2:].any()
    assert q[1, :3].tolist() == [0xFC, 0x70, 0x68]
    # E5M2: amax 1 -> e = -15 (code 112); 1 * 2^15 = 32768 = S.11110.00 (0x78)
    q5, s5 = orc.mx_quantize(x[:1], 1)
    assert s5.tolist() == [[112]] and q5[0, 0] == 0x78
    # a block maximum in [448, 512) saturates to 448 (its binade is 2^8)
    y = np.zeros((1, 32), np.float32)
    y[0, 0], y[0, 1] = 500.0, -1.0
    q, s = orc.mx_quantize(y, 0)
    assert s[0, 0] == 127 and q[0, 0] == 0x7E and q[0, 1] == 0xB8


def test_zero_block_and_errors(orc):
    x = np.zeros((1, 64), np.float32)
    x[0, 40] = 2.0
    q, s = orc.mx_quantize(x, 0)
    assert s[0, 0] == 0 and not q[0, :32].any()          # all-zero block: 2^-127, codes 0
    assert s[0, 1] == 127 + 1 - 8
    with pytest.raises(oracle.OracleError):
        orc.mx_quantize(np.ones((1, 48), np.float32), 0)
    bad = np.ones((1, 32), np.float32)
    bad[0, 3] = np.inf
    with pytest.raises(oracle.OracleError):
        orc.mx_quantize(bad, 0)


@pytest.mark.parametrize("fmt", [0, 1])
def test_scale_property_and_codes_vs_torch(orc, fmt):
    """For every block: 2^emax <= amax * 2^-e < 2^(emax+1) (the defining
    property, in float64), and the codes are PyTorch's cast of x * 2^-e
    wherever that is below the format's largest value (above it: saturated)."""
    x = workloads.randn_f32((64, 512), seed=71 + fmt)
    x *= np.float32(2.0) ** workloads.randint_f32((64, 512), 72, -20, 20)
    q, s = orc.mx_quantize(x, fmt)
    e = s.astype(np.int64) - 127
    blocks = np.abs(x.astype(np.float64)).reshape(64, 16, 32).max(axis=2)
    scaled = blocks * 2.0 ** (-e)
    assert np.all(scaled >= 2.0 ** EMAX[fmt]) and np.all(scaled < 2.0 ** (EMAX[fmt] + 1))
    y = (x.astype(np.float64).reshape(64, 16, 32) * 2.0 ** (-e)[:, :, None]).reshape(64, 512)
    assert np.array_equal(y.astype(np.float32).astype(np.float64), y)          # exact in fp32
    inr = np.abs(y) < MAXF[fmt]
    ref = torch.from_numpy(y.astype(np.float32)).to(TORCH_FP8[fmt]).view(torch.uint8).numpy()
    assert np.array_equal(q[inr], ref[inr])
    sat = 0x7E if fmt == 0 else 0x7B
    assert np.all((q[~inr] & 0x7F) == sat)


@pytest.mark.parametrize("fmt", [0, 1])
def test_power_of_two_invariance(orc, fmt):
    x = workloads.randn_f32((8, 256), seed=80)
    q0, s0 = orc.mx_quantize(x, fmt)
    for j in (-5, 3, 17):
        q, s = orc.mx_quantize(x * np.float32(2.0 ** j), fmt)
        assert np.array_equal(q, q0)
        assert np.array_equal(s.astype(int), s0.astype(int) + j)


def test_reconstruction_error_bound(orc):
    # Within E4M3's normal range after scaling, |X dec(q) - x| is at most half
    # a unit in the element's binade: relative <= 2^-4.  Scaled values above
    # 448 (the block maximum's binade reaches 512) saturate to 448 X.
    x = workloads.randn_f32((16, 256), seed=81)
    q, s = orc.mx_quantize(x, 0)
    X = np.repeat(orc.e8m0_decode(s), 32, axis=1)
    v = X * _dec(q, 0)
    y = np.abs(x) / X
    normal = (y >= 2.0 ** -6) & (y <= 448.0)
    assert np.all(np.abs(v - x)[normal] <= 2.0 ** -4 * np.abs(x)[normal] * (1 + 1e-12))
    over = y > 464.0
    assert np.array_equal(np.abs(v[over]), 448.0 * X[over])


@pytest.mark.parametrize("a_fmt,b_fmt", [(0, 0), (0, 1), (1, 1)])
def test_gemm_mx_vs_numpy(orc, a_fmt, b_fmt):
    M, N, K = 13, 9, 256
    A = workloads.random_codes((M, K), seed=90, fmt=a_fmt)
    B = workloads.random_codes((N, K), seed=91, fmt=b_fmt)
    g = torch.Generator().manual_seed(92)
    SA = torch.randint(110, 140, (M, K // 32), generator=g).to(torch.uint8).numpy()
    SB = torch.randint(110, 140, (N, K // 32), generator=g).to(torch.uint8).numpy()
    C = orc.gemm_mx(A, SA, B, SB, 0.5, a_fmt, b_fmt)
    XA = np.repeat(2.0 ** (SA.astype(np.float64) - 127), 32, axis=1)
    XB = np.repeat(2.0 ** (SB.astype(np.float64) - 127), 32, axis=1)
    ref = 0.5 * (XA * _dec(A, a_fmt)) @ (XB * _dec(B, b_fmt)).T
    np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-300)


def test_gemm_mx_quantised_close_to_fp32_product(orc):
    # end to end: block quantisation then the MX product approximates the
    # fp32 product.  Each operand element is off by at most 1/8 of its value
    # (2^-4 when not saturated, 1/8 at worst when a scaled value in
    # (448, 512) saturates) plus a subnormal remainder far below the block
    # scale, so |C - ref| <= (2/8 + 1/64) S elementwise; normwise the
    # rounding errors of both operands (each <= 2^-4 relative) stay below
    # 2^-4 of the product.
    x = workloads.randn_f32((32, 512), seed=93)
    w = workloads.randn_f32((24, 512), seed=94)
    qa, sa = orc.mx_quantize(x, 0)
    qb, sb = orc.mx_quantize(w, 0)
    C = orc.gemm_mx(qa, sa, qb, sb)
    ref = x.astype(np.float64) @ w.astype(np.float64).T
    S = np.abs(x.astype(np.float64)) @ np.abs(w.astype(np.float64)).T
    assert np.all(np.abs(C - ref) <= (2 / 8 + 1 / 64) * S)
    assert np.linalg.norm(C - ref) <= 2.0 ** -4 * np.linalg.norm(ref)
