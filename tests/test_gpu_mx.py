"""GPU parity of the block-scaled (MX) FP8 path against the oracle.

- fp8_quantize_mx: codes and E8M0 scales bit-exact against the oracle's
  mx_quantize (row-major scales) for E4M3 and E5M2, ragged shapes, zero
  blocks, huge, tiny and subnormal inputs; the tiled layout equals the
  oracle's scales placed by the header's layout formula (written out here).
- fp8_mx_scales_to_tiled: the oracle's row-major scales, tiled on the GPU.
- gemm_fp8_mx: structured cases first (scales varying by row group, by
  column group and by 32-element block, so a misplaced scale shows as a
  pattern), then small-integer inputs bit-exact against the FP64 oracle
  (every partial sum an integer below 2^24), then N(0,1) inputs within the
  FP32 / BF16 tolerances of tests/parity.py, all four format pairings, the
  swapped skinny path, and a large product checked on row/column blocks.
"""
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


def tiled_layout(sc_rowmajor, rows, cols):
    """The tiled scale layout of include/gb300fp8.h, from row-major scales."""
    kb = (cols + 127) // 128
    rt = (rows + 127) // 128
    out = np.full(rt * kb * 512, 127, np.uint8)
    r = np.arange(rows)[:, None]
    b = np.arange(cols // 32)[None, :]
    off = 512 * ((r // 128) * kb + b // 4) + 16 * (r % 32) + 4 * ((r % 128) // 32) + b % 4
    out[off] = sc_rowmajor
    return out


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _mx_inputs(rows, cols, seed):
    x = workloads.randn_f32((rows, cols), seed=seed)
    # vary the block magnitudes over many binades, with zero, tiny and huge blocks
    g = np.random.default_rng(seed)
    mag = 2.0 ** g.integers(-30, 30, size=(rows, cols // 32)).astype(np.float32)
    x = (x.reshape(rows, cols // 32, 32) * mag[:, :, None]).reshape(rows, cols).astype(np.float32)
    if rows > 2 and cols >= 96:
        x[0, :32] = 0.0                                   # an all-zero block
        x[0, 32:64] = -0.0
        x[1, 32:64] *= np.float32(2.0 ** -130)            # subnormal block
        x[2, 64:96] = np.float32(3.0e38)                  # near fp32 max
    return x


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("rows,cols", [(1, 32), (130, 160), (256, 512), (77, 4096), (300, 96)])
def test_mx_quantize_bit_exact(gb, orc, fmt, rows, cols):
    x = _mx_inputs(rows, cols, seed=rows * 7 + cols + fmt)
    q_ref, s_ref = orc.mx_quantize(x, fmt)
    xd = _dev(x)
    q, s = gb.fp8_quantize_mx(xd, fmt, scale_layout=0)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    assert np.array_equal(q.cpu().numpy(), q_ref)
    assert np.array_equal(s.cpu().numpy(), s_ref)
    q2, st = gb.fp8_quantize_mx(xd, fmt, scale_layout=1)
    torch.cuda.synchronize()
    assert np.array_equal(q2.cpu().numpy(), q_ref)
    assert np.array_equal(st.cpu().numpy(), tiled_layout(s_ref, rows, cols))
    # the layout converter gives the same tiled array from row-major scales
    st2 = gb.fp8_mx_scales_to_tiled(_dev(s_ref), rows, cols)
    torch.cuda.synchronize()
    assert np.array_equal(st2.cpu().numpy(), tiled_layout(s_ref, rows, cols))


def test_mx_quantize_rejects_nonfinite(gb):
    x = torch.zeros((4, 64), device="cuda")
    x[2, 40] = float("inf")
    gb.fp8_quantize_mx(x, 0)
    assert gb.fp8_last_device_error() == -4


def _gemm(gb, A, SA, B, SB, fmt=(0, 0), alpha=1.0, out_dtype=0):
    M, K = A.shape
    N = B.shape[0]
    C = gb.gemm_fp8_mx(_dev(A), _dev(tiled_layout(SA, M, K)), _dev(B), _dev(tiled_layout(SB, N, K)), alpha,
                       out_dtype, fmt[0], fmt[1])
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    return C.float().cpu().numpy()


ONE = 0x38          # E4M3 1.0


@pytest.mark.parametrize("case", ["a_rows", "a_blocks", "b_cols", "b_blocks"])
def test_mx_structured_scales(gb, orc, case):
    """All codes 1.0; scales 2^j with j set by A's row group, A's 32-element
    block, B's row (output column) group or B's block."""
    M, N, K = 256, 256, 256
    A = np.full((M, K), ONE, np.uint8)
    B = np.full((N, K), ONE, np.uint8)
    SA = np.full((M, K // 32), 127, np.uint8)
    SB = np.full((N, K // 32), 127, np.uint8)
    if case == "a_rows":
        SA += ((np.arange(M) // 32) % 8).astype(np.uint8)[:, None]
    elif case == "a_blocks":
        SA += (np.arange(K // 32) % 8).astype(np.uint8)[None, :]
    elif case == "b_cols":
        SB += ((np.arange(N) // 32) % 8).astype(np.uint8)[:, None]
    else:
        SB += (np.arange(K // 32) % 8).astype(np.uint8)[None, :]
    C = _gemm(gb, A, SA, B, SB)
    ref = orc.gemm_mx(A, SA, B, SB)
    assert np.array_equal(C.astype(np.float64), ref), (C[::32, ::32], ref[::32, ::32])


@pytest.mark.parametrize("fmt", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (200, 72, 320), (128, 384, 1024), (16, 512, 2048),
                                   (300, 130, 4096)])
def test_mx_small_integers_bit_exact(gb, orc, fmt, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + K, fmt=fmt[0])
    B = workloads.small_int_codes((N, K), seed=N + K + 1, fmt=fmt[1])
    g = np.random.default_rng(M * N + K)
    SA = g.integers(127, 129, size=(M, K // 32)).astype(np.uint8)      # scales 1 or 2
    SB = g.integers(126, 128, size=(N, K // 32)).astype(np.uint8)      # scales 1/2 or 1
    C = _gemm(gb, A, SA, B, SB, fmt)
    ref = orc.gemm_mx(A, SA, B, SB, a_fmt=fmt[0], b_fmt=fmt[1])
    assert np.array_equal(C.astype(np.float64), ref)


@pytest.mark.parametrize("fmt", [(0, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (1000, 600, 1024), (64, 2048, 1024), (512, 512, 4096)])
def test_mx_normal_inputs(gb, orc, fmt, M, N, K):
    x = workloads.randn_f32((M, K), seed=M + 3)
    w = workloads.randn_f32((N, K), seed=N + 4)
    A, SA = orc.mx_quantize(x, fmt[0])
    B, SB = orc.mx_quantize(w, fmt[1])
    ref = orc.gemm_mx(A, SA, B, SB, alpha=0.75, a_fmt=fmt[0], b_fmt=fmt[1])
    C = _gemm(gb, A, SA, B, SB, fmt, alpha=0.75, out_dtype=0)
    parity.check_fp32(C, ref)
    Cb = _gemm(gb, A, SA, B, SB, fmt, alpha=0.75, out_dtype=1)
    S = orc.gemm_mx(parity.abs_codes(A), SA, parity.abs_codes(B), SB, alpha=0.75, a_fmt=fmt[0],
                    b_fmt=fmt[1])
    parity.check_bf16(Cb, ref, S, K)


@pytest.mark.parametrize("M,N,K", [(1024, 1024, 1024), (16, 4096, 4096)])
def test_mx_pipeline_quantized_on_gpu(gb, orc, M, N, K):
    """fp32 -> fp8_quantize_mx (tiled scales) -> gemm_fp8_mx on the GPU,
    against the oracle's quantisation and product."""
    x = workloads.randn_f32((M, K), seed=11)
    w = workloads.randn_f32((N, K), seed=12)
    A, SAt = gb.fp8_quantize_mx(_dev(x), 0, scale_layout=1)
    B, SBt = gb.fp8_quantize_mx(_dev(w), 0, scale_layout=1)
    C = gb.gemm_fp8_mx(A, SAt, B, SBt, 1.0, gb.OUT_F32)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    Ao, SAo = orc.mx_quantize(x, 0)
    Bo, SBo = orc.mx_quantize(w, 0)
    assert np.array_equal(A.cpu().numpy(), Ao) and np.array_equal(B.cpu().numpy(), Bo)
    parity.check_fp32(C.cpu().numpy(), orc.gemm_mx(Ao, SAo, Bo, SBo))


def test_mx_large_blocks(gb, orc):
    """8192^3 on the GPU; the oracle takes the first and last 128 rows of A
    against the first and last 128 rows of B (four 128 x 128 blocks)."""
    M = N = K = 8192
    x = workloads.randn_f32((M, K), seed=21)
    w = workloads.randn_f32((N, K), seed=22)
    A, SAt = gb.fp8_quantize_mx(_dev(x), 0, scale_layout=1)
    B, SBt = gb.fp8_quantize_mx(_dev(w), 0, scale_layout=1)
    C = gb.gemm_fp8_mx(A, SAt, B, SBt, 1.0, gb.OUT_BF16)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    C = C.float().cpu().numpy()
    rows = np.r_[0:128, M - 128:M]
    Ao, SAo = orc.mx_quantize(x[rows], 0)
    Bo, SBo = orc.mx_quantize(w[rows], 0)
    ref = orc.gemm_mx(Ao, SAo, Bo, SBo)
    S = orc.gemm_mx(parity.abs_codes(Ao), SAo, parity.abs_codes(Bo), SBo)
    parity.check_bf16(C[np.ix_(rows, rows)], ref, S, K)


# Shapes whose N tiles are 256 wide (the planner keeps 256 while 2 x row
# blocks x column blocks reach the SM count): one accumulator, B's scales
# in two 128-row chunks per k-block, ring after the accumulator.  N = 800
# leaves the last tile's second 128-row scale chunk outside B (not loaded).
WIDE = [(4096, 1024, 256), (4096, 1000, 640), (4096, 800, 1024)]


def test_mx_wide_tiles_are_planned(gb):
    for M, N, K in WIDE:
        info = gb.gemm_fp8_mx_plan(M, N, K)
        assert info["mt"] == 1 and info["bn"] == 256 and info["cluster"] == 0, (M, N, K, info)
    assert gb.gemm_fp8_mx_plan(1024, 1024, 1024)["bn"] == 128


@pytest.mark.parametrize("case", ["a_rows", "a_blocks", "b_cols", "b_blocks"])
def test_mx_wide_tiles_structured_scales(gb, orc, case):
    M, N, K = 4096, 1024, 256
    A = np.full((M, K), ONE, np.uint8)
    B = np.full((N, K), ONE, np.uint8)
    SA = np.full((M, K // 32), 127, np.uint8)
    SB = np.full((N, K // 32), 127, np.uint8)
    if case == "a_rows":
        SA += ((np.arange(M) // 32) % 8).astype(np.uint8)[:, None]
    elif case == "a_blocks":
        SA += (np.arange(K // 32) % 8).astype(np.uint8)[None, :]
    elif case == "b_cols":
        SB += ((np.arange(N) // 32) % 8).astype(np.uint8)[:, None]
    else:
        SB += (np.arange(K // 32) % 8).astype(np.uint8)[None, :]
    C = _gemm(gb, A, SA, B, SB)
    rows = np.r_[0:160, M - 160:M]
    ref = orc.gemm_mx(A[rows], SA[rows], B, SB)
    assert np.array_equal(C[rows].astype(np.float64), ref), (C[rows][::32, ::32], ref[::32, ::32])


@pytest.mark.parametrize("fmt", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", WIDE)
def test_mx_wide_tiles_small_integers_bit_exact(gb, orc, fmt, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + K + 3, fmt=fmt[0])
    B = workloads.small_int_codes((N, K), seed=N + K + 4, fmt=fmt[1])
    g = np.random.default_rng(M + N + K)
    SA = g.integers(127, 129, size=(M, K // 32)).astype(np.uint8)
    SB = g.integers(126, 128, size=(N, K // 32)).astype(np.uint8)
    C = _gemm(gb, A, SA, B, SB, fmt)
    rows = np.r_[0:128, 1900:2100, M - 128:M]
    ref = orc.gemm_mx(A[rows], SA[rows], B, SB, a_fmt=fmt[0], b_fmt=fmt[1])
    assert np.array_equal(C[rows].astype(np.float64), ref)


@pytest.mark.parametrize("M,N,K", WIDE)
def test_mx_wide_tiles_normal_inputs(gb, orc, M, N, K):
    x = workloads.randn_f32((M, K), seed=M + 13)
    w = workloads.randn_f32((N, K), seed=N + 14)
    A, SA = orc.mx_quantize(x, 0)
    B, SB = orc.mx_quantize(w, 0)
    rows = np.r_[0:128, M - 256:M]
    ref = orc.gemm_mx(A[rows], SA[rows], B, SB, alpha=0.5)
    C = _gemm(gb, A, SA, B, SB, alpha=0.5, out_dtype=0)
    parity.check_fp32(C[rows], ref)
    Cb = _gemm(gb, A, SA, B, SB, alpha=0.5, out_dtype=1)
    S = orc.gemm_mx(parity.abs_codes(A[rows]), SA[rows], parity.abs_codes(B), SB, alpha=0.5)
    parity.check_bf16(Cb[rows], ref, S, K)


# CTA pairs (256 x 256 tiles over two CTAs, each holding its 128 rows of A
# and of B, their scale chunks loaded by TMA into each CTA's tensor memory):
# problems whose 256-row tiles fill the SMs.  Ragged N and M put part of the
# odd CTA's half outside B or A.
PAIRS = [(4096, 2048, 256), (4096, 2000, 640), (4000, 2048, 1024)]


def test_mx_pairs_are_planned(gb):
    for M, N, K in PAIRS + [(8192, 8192, 8192)]:
        info = gb.gemm_fp8_mx_plan(M, N, K)
        assert info["mt"] == 3 and info["bn"] == 256 and info["cluster"] == 2, (M, N, K, info)


@pytest.mark.parametrize("case", ["a_rows", "a_blocks", "b_cols", "b_blocks"])
def test_mx_pairs_structured_scales(gb, orc, case):
    M, N, K = PAIRS[0]
    A = np.full((M, K), ONE, np.uint8)
    B = np.full((N, K), ONE, np.uint8)
    SA = np.full((M, K // 32), 127, np.uint8)
    SB = np.full((N, K // 32), 127, np.uint8)
    if case == "a_rows":
        SA += ((np.arange(M) // 32) % 8).astype(np.uint8)[:, None]
    elif case == "a_blocks":
        SA += (np.arange(K // 32) % 8).astype(np.uint8)[None, :]
    elif case == "b_cols":
        SB += ((np.arange(N) // 32) % 8).astype(np.uint8)[:, None]
    else:
        SB += (np.arange(K // 32) % 8).astype(np.uint8)[None, :]
    C = _gemm(gb, A, SA, B, SB)
    rows = np.r_[0:288, M - 160:M]
    ref = orc.gemm_mx(A[rows], SA[rows], B, SB)
    assert np.array_equal(C[rows].astype(np.float64), ref), (C[rows][::32, ::32], ref[::32, ::32])


@pytest.mark.parametrize("fmt", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", PAIRS)
def test_mx_pairs_small_integers_bit_exact(gb, orc, fmt, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M + K + 5, fmt=fmt[0])
    B = workloads.small_int_codes((N, K), seed=N + K + 6, fmt=fmt[1])
    g = np.random.default_rng(M + 2 * N + K)
    SA = g.integers(127, 129, size=(M, K // 32)).astype(np.uint8)
    SB = g.integers(126, 128, size=(N, K // 32)).astype(np.uint8)
    C = _gemm(gb, A, SA, B, SB, fmt)
    rows = np.r_[0:300, 1900:2100, M - 300:M]
    ref = orc.gemm_mx(A[rows], SA[rows], B, SB, a_fmt=fmt[0], b_fmt=fmt[1])
    assert np.array_equal(C[rows].astype(np.float64), ref)


@pytest.mark.parametrize("M,N,K", PAIRS)
def test_mx_pairs_normal_inputs(gb, orc, M, N, K):
    x = workloads.randn_f32((M, K), seed=M + 23)
    w = workloads.randn_f32((N, K), seed=N + 24)
    A, SA = orc.mx_quantize(x, 0)
    B, SB = orc.mx_quantize(w, 0)
    rows = np.r_[0:256, M - 256:M]
    ref = orc.gemm_mx(A[rows], SA[rows], B, SB, alpha=0.5)
    C = _gemm(gb, A, SA, B, SB, alpha=0.5, out_dtype=0)
    parity.check_fp32(C[rows], ref)
    Cb = _gemm(gb, A, SA, B, SB, alpha=0.5, out_dtype=1)
    S = orc.gemm_mx(parity.abs_codes(A[rows]), SA[rows], parity.abs_codes(B), SB, alpha=0.5)
    parity.check_bf16(Cb[rows], ref, S, K)


def test_mx_pairs_stalled_launch_times_out(gb):
    """The failure path on block-scaled pairs: loads withheld, every wait
    bounded (50 ms here), FP8_ERR_TIMEOUT recorded, C unwritten, and the
    next launch exact."""
    M, N, K = PAIRS[0]
    A = workloads.small_int_codes((M, K), seed=41)
    B = workloads.small_int_codes((N, K), seed=42)
    SA = np.full((M, K // 32), 127, np.uint8)
    SB = np.full((N, K // 32), 128, np.uint8)
    ref = _gemm(gb, A, SA, B, SB)
    At, Bt = _dev(A), _dev(B)
    SAt, SBt = _dev(tiled_layout(SA, M, K)), _dev(tiled_layout(SB, N, K))
    C = torch.full((M, N), float("nan"), device="cuda")
    gb.fp8_test_stall_gemm_loads(1, 50.0)
    try:
        gb.gemm_fp8_mx(At, SAt, Bt, SBt, 1.0, gb.OUT_F32, C=C)
        assert gb.fp8_last_device_error() == -7
    finally:
        gb.fp8_test_stall_gemm_loads(0, 0.0)
    assert torch.isnan(C).all()
    gb.gemm_fp8_mx(At, SAt, Bt, SBt, 1.0, gb.OUT_F32, C=C)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    assert np.array_equal(C.cpu().numpy(), ref)
