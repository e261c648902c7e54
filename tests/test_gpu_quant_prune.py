"""GPU parity: fp8_quantize_e4m3_prune24 (per-row E4M3 quantisation and the
2:4 compression of its codes in one pass) against the oracle's quantise then
prune, and against the two separate kernels, bit for bit: codes, scales,
kept codes and metadata."""
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


def _fused(gb, xt):
    out = gb.fp8_quantize_e4m3_prune24(xt)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    return [t.cpu().numpy() for t in out]


def _check_oracle(orc, x, got):
    q, d, v, m = got
    qo, do = orc.quantize(x, 1)
    vo, mo = orc.prune24(qo)
    assert np.array_equal(d, do)
    assert np.array_equal(q, qo)
    assert np.array_equal(v, vo)
    assert np.array_equal(m, mo)


# one 128-column row, a few rows, a ragged row count, the benchmark's row
# length (16384), a K with an odd number of 128-column blocks
@pytest.mark.parametrize("shape", [(1, 128), (3, 256), (257, 1024), (64, 16384), (1000, 4224)])
def test_equals_oracle(gb, orc, shape):
    x = workloads.randn_f32(shape, seed=shape[0] * 7 + shape[1])
    _check_oracle(orc, x, _fused(gb, torch.from_numpy(x).cuda()))


def test_ties_zeros_and_signed_zeros(gb, orc):
    """Groups of equal magnitudes (kept: the two lowest indices), signed
    zeros, all-zero rows (scale 1, codes of the zeros), a lone non-zero."""
    x = np.zeros((6, 128), np.float32)
    x[0] = np.tile(np.array([1.0, -1.0, 1.0, -1.0], np.float32), 32)
    x[1] = np.tile(np.array([-0.0, 0.0, -0.0, 2.0], np.float32), 32)
    x[2] = -0.0
    x[4, 77] = -3.0
    x[5] = np.tile(np.array([0.5, 448.0, 0.5, -448.0], np.float32), 32)
    _check_oracle(orc, x, _fused(gb, torch.from_numpy(x).cuda()))


def test_strided_rows(gb, orc):
    wide = workloads.randn_f32((40, 1024 + 64), seed=5)
    xt = torch.from_numpy(wide).cuda()[:, 32:32 + 1024]         # ldx 1088, 16-byte aligned start
    qbuf = torch.zeros((40, 1024 + 128), dtype=torch.uint8, device="cuda")
    q, d, v, m = gb.fp8_quantize_e4m3_prune24(xt, q=qbuf[:, :1024])
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    _check_oracle(orc, wide[:, 32:32 + 1024], [t.cpu().numpy() for t in (q, d, v, m)])
    assert torch.count_nonzero(qbuf[:, 1024:]) == 0              # nothing past each row


def test_equals_separate_kernels_full_size(gb):
    """The benchmark's A operand (16384 x 16384 fp32): the fused pass equals
    fp8_quantize_e4m3(x, 1) followed by prune24_compress, bit for bit."""
    g = torch.Generator(device="cuda").manual_seed(workloads.SEED_A)
    x = torch.randn((16384, 16384), generator=g, device="cuda")
    q, d, v, m = gb.fp8_quantize_e4m3_prune24(x)
    q2, d2 = gb.fp8_quantize_e4m3(x, 1)
    v2, m2 = gb.prune24_compress(q2)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    assert torch.equal(d, d2) and torch.equal(q, q2)
    assert torch.equal(v, v2) and torch.equal(m, m2)


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_reported(gb, bad):
    x = np.ones((8, 256), np.float32)
    x[3, 9] = bad
    gb.fp8_quantize_e4m3_prune24(torch.from_numpy(x).cuda())
    assert gb.fp8_last_device_error() == -4          # FP8_ERR_NONFINITE
    assert gb.fp8_last_device_error() == 0


def test_shape_and_alignment_rejected(gb):
    with pytest.raises(gb.Fp8Error):
        gb.fp8_quantize_e4m3_prune24(torch.ones((4, 100), device="cuda"))
    wide = torch.ones((4, 260), device="cuda")
    with pytest.raises(gb.Fp8Error):
        gb.fp8_quantize_e4m3_prune24(wide[:, 1:257])                # x not 16-byte aligned
