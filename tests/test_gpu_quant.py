"""GPU parity: fp8_quantize_e4m3 (scale selection + E4M3 encode) against the
oracle, bit-exact on codes and scales."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


def _run(gb, x: np.ndarray, mode: int):
    xt = torch.from_numpy(x).cuda()
    q, d = gb.fp8_quantize_e4m3(xt, mode)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    return q.cpu().numpy(), d.cpu().numpy()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (33, 3), (256, 256), (257, 1000), (64, 4096),
                                   (1000, 1029)])
def test_parity_small(gb, orc, mode, shape):
    x = workloads.randn_f32(shape, seed=shape[0] + 10 * shape[1])
    q, d = _run(gb, x, mode)
    qo, do = orc.quantize(x, mode)
    assert np.array_equal(q, qo)
    assert np.array_equal(d, do)


@pytest.mark.parametrize("mode", [0, 1])
def test_parity_full_size(gb, orc, mode):
    # the square-sweep operand size used by the benchmark (8192 x 8192 fp32)
    x = workloads.randn_f32((8192, 8192), seed=workloads.SEED_A)
    q, d = _run(gb, x, mode)
    qo, do = orc.quantize(x, mode)
    assert np.array_equal(d, do)
    assert np.array_equal(q, qo)


def test_strided_rows(gb, orc):
    wide = workloads.randn_f32((40, 100), seed=3)
    xt = torch.from_numpy(wide).cuda()[:, 7:67]       # ld = 100, unaligned start
    q, d = gb.fp8_quantize_e4m3(xt, 1)
    qo, do = orc.quantize(wide[:, 7:67], 1)
    assert np.array_equal(q.cpu().numpy(), qo) and np.array_equal(d.cpu().numpy(), do)


def test_zero_rows(gb):
    x = np.zeros((4, 64), np.float32)
    x[2, 5] = -3.0
    q, d = _run(gb, x, 1)
    assert np.array_equal(d, np.array([1, 1, 3 / 448, 1], np.float32))
    assert np.all(q[[0, 1, 3]] == 0) and q[2, 5] == 0xFE


@pytest.mark.parametrize("bad", [np.nan, np.inf])
@pytest.mark.parametrize("mode", [0, 1])
def test_nonfinite_reported(gb, mode, bad):
    x = np.ones((8, 64), np.float32)
    x[3, 9] = bad
    xt = torch.from_numpy(x).cuda()
    gb.fp8_quantize_e4m3(xt, mode)
    assert gb.fp8_last_device_error() == -4          # FP8_ERR_NONFINITE
    assert gb.fp8_last_device_error() == 0           # cleared by the read


def test_device_encoder_all_in_range_fp32(gb, orc):
    """Every fp32 bit pattern with |x| <= 448 through the device encoder.

    A tensor whose amax is exactly 448 gets s = 448/448 = 1, so the codes are
    enc(x) itself; each chunk carries a sentinel row of 448."""
    top = 0x43E00000                                     # bits of 448.0f
    chunk = 1 << 26
    cols = 1024
    for sign in (0, 0x80000000):
        for lo in range(0, top + 1, chunk):
            hi = min(lo + chunk, top + 1)
            n = hi - lo
            rows = (n + cols - 1) // cols
            bits = torch.arange(lo, lo + rows * cols, dtype=torch.int64, device="cuda")
            bits = torch.clamp(bits, max=hi - 1) | sign
            bits = torch.where(bits >= 2 ** 31, bits - 2 ** 32, bits)     # as signed int32
            x = bits.to(torch.int32).view(torch.float32).reshape(rows, cols)
            x = torch.cat([x, torch.full((1, cols), 448.0, device="cuda")])
            q, d = gb.fp8_quantize_e4m3(x, 0)
            assert d.item() == 1.0
            got = q[:-1].reshape(-1)[:n].cpu().numpy()
            ref = orc.encode_pattern_range(lo | sign, (hi - 1 | sign) + 1)
            assert np.array_equal(got, ref), f"chunk at {lo | sign:#x}"
