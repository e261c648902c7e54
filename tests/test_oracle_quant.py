"""Pins for the oracle's quantisation (scale selection + E4M3 encode).

Checked against: hand-worked closed-form cases (tests/golden), an independent
restatement through PyTorch library ops (amax, fp32 divide and multiply, the
float8_e4m3fn cast), and invariants (amax maps to +-448, power-of-two scaling
leaves the codes unchanged, per-row = per-tensor on each row).
"""
import os

import numpy as np
import pytest
import torch

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cases():
    out = []
    with open(os.path.join(GOLDEN, "quantize_closed_form.txt")) as f:
        for line in f:
            if line.startswith("case"):
                xs, codes, d = line[4:].split("|")
                out.append((np.array([float(v) for v in xs.split()], np.float32),
                            np.array([int(c, 16) for c in codes.split()], np.uint8),
                            float(d)))
    return out


def test_closed_form_cases(orc):
    cases = _cases()
    assert len(cases) == 2
    for x, codes, d in cases:
        q, dq = orc.quantize(x[None, :], 0)
        assert np.array_equal(q[0], codes)
        assert dq[0] == np.float32(d)


def _torch_quantize(x: np.ndarray, mode: int):
    t = torch.from_numpy(x)
    amax = t.abs().amax() if mode == 0 else t.abs().amax(dim=1, keepdim=True)
    amax = torch.as_tensor(amax, dtype=torch.float32)
    one = torch.ones_like(amax)
    c448 = torch.full_like(amax, 448.0)
    s = torch.where(amax == 0, one, c448 / amax)
    d = torch.where(amax == 0, one, amax / c448)
    y = t * s                                 # one fp32 multiply, |y| <= 448
    q = y.to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    return q, d.reshape(-1).numpy()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("shape", [(1, 1), (3, 17), (64, 256), (257, 96)])
def test_matches_torch_restatement(orc, mode, shape):
    x = workloads.randn_f32(shape, seed=shape[0] * 7 + shape[1])
    q, d = orc.quantize(x, mode)
    qt, dt = _torch_quantize(x, mode)
    assert np.array_equal(q, qt)
    assert np.array_equal(d, dt)


def test_amax_maps_to_448(orc):
    x = workloads.randn_f32((33, 130), seed=5)
    q, _ = orc.quantize(x, 1)
    for r in range(x.shape[0]):
        i = np.argmax(np.abs(x[r]))
        assert q[r, i] == (0xFE if x[r, i] < 0 else 0x7E)
    q0, _ = orc.quantize(x, 0)
    i = np.unravel_index(np.argmax(np.abs(x)), x.shape)
    assert q0[i] & 0x7F == 0x7E


def test_power_of_two_invariance(orc):
    x = workloads.randn_f32((16, 64), seed=6)
    for mode in (0, 1):
        q, d = orc.quantize(x, mode)
        for k in (-3, 5):
            q2, d2 = orc.quantize(x * np.float32(2.0 ** k), mode)
            assert np.array_equal(q, q2)
            assert np.array_equal(d2, d * np.float32(2.0 ** k))


def test_rows_independent(orc):
    x = workloads.randn_f32((9, 40), seed=7)
    q, d = orc.quantize(x, 1)
    for r in range(9):
        qr, dr = orc.quantize(x[r:r + 1], 0)
        assert np.array_equal(q[r], qr[0]) and d[r] == dr[0]


def test_nearest_code(orc):
    # each code is a nearest finite E4M3 value to fl32(x * s)
    x = workloads.randn_f32((8, 300), seed=8)
    q, d = orc.quantize(x, 1)
    s = (np.float32(448.0) / np.abs(x).max(axis=1, keepdims=True)).astype(np.float32)
    y = (x * s).astype(np.float64)
    table = orc.e4m3_decode(np.arange(0x7F, dtype=np.uint8))
    v = orc.e4m3_decode(q)
    best = np.min(np.abs(np.abs(y)[..., None] - table[None, None, :]), axis=-1)
    assert np.array_equal(np.abs(v - y), best)


def test_zero_tensor(orc):
    q, d = orc.quantize(np.zeros((4, 8), np.float32), 0)
    assert np.all(q == 0) and d[0] == 1.0
    q, d = orc.quantize(np.zeros((4, 8), np.float32), 1)
    assert np.all(q == 0) and np.all(d == 1.0)


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_rejected(orc, bad):
    x = np.ones((2, 4), np.float32)
    x[1, 2] = bad
    with pytest.raises(oracle.OracleError):
        orc.quantize(x, 0)
    with pytest.raises(oracle.OracleError):
        orc.quantize(x, 1)
