"""GPU parity: gemm_fp8_dense (and the grouped launch) against the FP64 oracle.

Exact cases (small-integer codes: every partial sum is an integer far below
2^24) must match bit for bit in FP32 output; N(0,1) cases are checked with
the tolerances in tests/parity.py; full-size shapes are checked on seeded
sampled entries plus two full rows and two full columns.
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _codes(a):
    """Device copy of a code matrix with its row stride padded to a multiple
    of 16 bytes (the TMA row-stride rule); the view has the original shape."""
    M, K = a.shape
    ld = max(16, (K + 15) // 16 * 16)
    t = torch.zeros((M, ld), dtype=torch.uint8, device="cuda")
    t[:, :K] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t[:, :K]


def _ones(n=1):
    return torch.ones(n, dtype=torch.float32, device="cuda")


def _gemm(gb, A, B, dA, a_mode, dB, b_mode, alpha, out_dtype):
    C = gb.gemm_fp8_dense(_codes(A), _codes(B), _cuda(dA), a_mode, _cuda(dB), b_mode, alpha,
                          out_dtype)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    return C.float().cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (128, 256, 128), (200, 72, 320),
                                   (16, 512, 1024), (1, 1, 1), (300, 17, 4100)])
def test_small_integers_bit_exact(gb, orc, M, N, K):
    A = workloads.small_int_codes((M, K), seed=M)
    B = workloads.small_int_codes((N, K), seed=N + 1)
    one = np.ones(1, np.float32)
    C = _gemm(gb, A, B, one, 0, one, 0, 1.0, gb.OUT_F32)
    ref = orc.gemm(A, B, one, 0, one, 0)
    assert np.array_equal(C.astype(np.float64), ref)


def _quantized(M, N, K, a_mode, b_mode, orc, seed=0):
    x = workloads.randn_f32((M, K), seed=workloads.SEED_A + seed)
    w = workloads.randn_f32((N, K), seed=workloads.SEED_B + seed)
    A, dA = orc.quantize(x, a_mode)
    B, dB = orc.quantize(w, b_mode)
    return A, dA, B, dB


def test_dense_256_fp32_per_tensor(gb, orc):
    """The 256^3 single-call case: per-tensor scales, FP32 output."""
    A, dA, B, dB = _quantized(256, 256, 256, 0, 0, orc)
    C = _gemm(gb, A, B, dA, 0, dB, 0, 1.0, gb.OUT_F32)
    ref = orc.gemm(A, B, dA, 0, dB, 0)
    parity.check_fp32(C, ref)


@pytest.mark.parametrize("M,N,K", [(1024, 1024, 1024), (1000, 1500, 700), (16, 8192, 1024),
                                   (64, 3000, 512), (128, 1024, 2048), (129, 333, 256)])
def test_dense_bf16_per_row(gb, orc, M, N, K):
    A, dA, B, dB = _quantized(M, N, K, 1, 1, orc, seed=M)
    C = _gemm(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16)
    ref = orc.gemm(A, B, dA, 1, dB, 1)
    S = orc.gemm(parity.abs_codes(A), parity.abs_codes(B), dA, 1, dB, 1)
    parity.check_bf16(C, ref, S, K)


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (500, 300, 1000)])
def test_dense_fp32_per_row_alpha(gb, orc, M, N, K):
    A, dA, B, dB = _quantized(M, N, K, 1, 1, orc, seed=3)
    C = _gemm(gb, A, B, dA, 1, dB, 1, -0.625, gb.OUT_F32)
    parity.check_fp32(C, orc.gemm(A, B, dA, 1, dB, 1, -0.625))


def _sampled_check(gb, orc, M, N, K, out_dtype, seed=0):
    A, dA, B, dB = _quantized(M, N, K, 1, 1, orc, seed=seed)
    C = _gemm(gb, A, B, dA, 1, dB, 1, 1.0, out_dtype)
    ms, ns = workloads.sample_pairs(M, N, 4096, seed=99)
    rows = np.array([0, M - 1])
    cols = np.array([0, N - 1])
    ms = np.concatenate([ms, np.repeat(rows, N), np.tile(np.arange(M), 2)])
    ns = np.concatenate([ns, np.tile(np.arange(N), 2), np.repeat(cols, M)])
    ref = orc.gemm_sampled(A, B, dA, 1, dB, 1, 1.0, ms, ns)
    S = orc.gemm_sampled(parity.abs_codes(A), parity.abs_codes(B), dA, 1, dB, 1, 1.0, ms, ns)
    got = C[ms, ns]
    if out_dtype == gb.OUT_BF16:
        parity.check_bf16(got, ref, S, K)
    else:
        parity.check_fp32(got, ref)


@pytest.mark.parametrize("M,N,K", [(8192, 8192, 8192), (16, 8192, 8192), (128, 8192, 8192)])
def test_full_size_sampled(gb, orc, M, N, K):
    _sampled_check(gb, orc, M, N, K, gb.OUT_BF16)


def test_identity(gb, orc):
    K = 256
    A = workloads.random_codes((300, K), seed=5)
    one = torch.tensor([1.0]).to(torch.float8_e4m3fn).view(torch.uint8).item()
    I = np.zeros((K, K), np.uint8)
    I[np.arange(K), np.arange(K)] = one
    s = np.ones(1, np.float32)
    C = _gemm(gb, A, I, s, 0, s, 0, 1.0, gb.OUT_F32)
    assert np.array_equal(C.astype(np.float64), orc.e4m3_decode(A))


def test_row_permutation_bitwise(gb, orc):
    A, dA, B, dB = _quantized(384, 256, 512, 1, 1, orc, seed=7)
    C = _gemm(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_F32)
    # permute whole 128-row tiles so each row keeps its accumulation order
    perm = np.concatenate([np.arange(256, 384), np.arange(0, 128), np.arange(128, 256)])
    Cp = _gemm(gb, A[perm], B, dA[perm], 1, dB, 1, 1.0, gb.OUT_F32)
    assert np.array_equal(Cp, C[perm])


def test_k_zero_writes_zeros(gb):
    C = torch.full((5, 7), 3.0, device="cuda")
    gb.gemm_fp8_dense(torch.empty((5, 0), dtype=torch.uint8, device="cuda"),
                      torch.empty((7, 0), dtype=torch.uint8, device="cuda"), _ones(), 0, _ones(),
                      0, 1.0, gb.OUT_F32, C=C)
    assert torch.count_nonzero(C).item() == 0


def test_misaligned_ld_rejected(gb):
    A = torch.zeros((4, 40), dtype=torch.uint8, device="cuda")[:, :36]
    B = torch.zeros((4, 36), dtype=torch.uint8, device="cuda")
    with pytest.raises(gb.Fp8Error) as e:
        gb.gemm_fp8_dense(A, B, _ones(), 0, _ones(), 0)
    assert e.value.status == -3


def test_grouped_equals_single_bitwise(gb, orc):
    shapes = [(512, 768, 1024), (16, 2048, 512), (300, 200, 256), (1024, 256, 4096)]
    probs, outs, singles, keep = [], [], [], []
    for i, (M, N, K) in enumerate(shapes):
        A, dA, B, dB = _quantized(M, N, K, 1, 1, orc, seed=20 + i)
        t = [_cuda(A), _cuda(B), _cuda(dA), _cuda(dB)]
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        keep += t
        outs.append(C)
        probs.append(gb.make_problem(t[0], t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16))
        singles.append(gb.gemm_fp8_dense(t[0], t[1], t[2], 1, t[3], 1, 1.0, gb.OUT_BF16))
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    for C, Cs in zip(outs, singles):
        assert torch.equal(C, Cs)


@pytest.fixture()
def tile_cfg(gb):
    yield gb.fp8_gemm_set_tile_config
    gb.fp8_gemm_set_tile_config(0, 0)


@pytest.mark.parametrize("M,N,K", [(256, 256, 256), (300, 520, 700), (1000, 1500, 1024),
                                   (16, 1024, 512), (129, 256, 4100)])
@pytest.mark.parametrize("gm", [0, 1, 3])
def test_tile_configs_bitwise_equal_and_correct(gb, orc, tile_cfg, M, N, K, gm):
    """256-row tiles (mt=2) and 128-row tiles (mt=1), any raster band height:
    the same per-element K order, so bitwise equal results."""
    A, dA, B, dB = _quantized(M, N, K, 1, 1, orc, seed=M + N)
    outs = []
    for mt in (1, 2):
        tile_cfg(mt, gm)
        outs.append(_gemm(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_F32))
    assert np.array_equal(outs[0], outs[1])
    parity.check_fp32(outs[1], orc.gemm(A, B, dA, 1, dB, 1))


@pytest.mark.parametrize("M,N,K", [(16, 4096, 4096), (1, 8192, 4096), (40, 2048, 8192),
                                   (1024, 1024, 1024), (100, 300, 2000)])
def test_split_k_repeatable_and_correct(gb, orc, M, N, K):
    """Few 128-row tiles: K is split across CTAs (partials in the stream's
    workspace, the last unit of each tile adds them in slice order).  Calls
    repeat bit for bit (the tile counters reset themselves) and match the
    oracle."""
    A, dA, B, dB = _quantized(M, N, K, 1, 1, orc, seed=M + 5)
    C1 = _gemm(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16)
    C2 = _gemm(gb, A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16)
    assert np.array_equal(C1, C2)
    ref = orc.gemm(A, B, dA, 1, dB, 1)
    S = orc.gemm(parity.abs_codes(A), parity.abs_codes(B), dA, 1, dB, 1)
    parity.check_bf16(C1, ref, S, K)


def test_split_k_workspace_reuse_streams_and_capture(gb, orc):
    """Split launches share their stream's persistent workspace.  A sequence
    that grows and shrinks it, the same calls on a second stream, and a
    captured graph (which owns a workspace of its own, freed after the graph
    is destroyed) all give the bitwise-same results as the first calls."""
    shapes = [(8, 4096, 4096), (16, 8192, 8192), (8, 4096, 4096), (1, 2048, 4096)]
    data = []
    for i, (M, N, K) in enumerate(shapes):
        A = _codes(workloads.random_codes((M, K), seed=300 + i))
        B = _codes(workloads.random_codes((N, K), seed=400 + i))
        data.append((A, B, _ones(M), _ones(N)))

    def run(outs=None, stream=None):
        outs = outs or [None] * len(data)
        return [gb.gemm_fp8_dense(A, B, sa, 1, sb, 1, 1.0, gb.OUT_F32, C=o, stream=stream)
                for (A, B, sa, sb), o in zip(data, outs)]

    first = run()
    torch.cuda.synchronize()
    for f in first:
        assert not torch.isnan(f).any()
    for o, f in zip(run(), first):
        assert torch.equal(o, f)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        on_side = run(stream=side)
    side.synchronize()
    for o, f in zip(on_side, first):
        assert torch.equal(o, f)
    outs = [torch.empty_like(f) for f in first]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run(outs)
    for _ in range(2):
        for o in outs:
            o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for o, f in zip(outs, first):
            assert torch.equal(o, f)
    del g                                  # releases the graph's workspace
    torch.cuda.synchronize()
    for o, f in zip(run(), first):         # the next split launch frees it
        assert torch.equal(o, f)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    A, B = data[0][0].cpu().numpy(), data[0][1].cpu().numpy()
    one = np.ones(1, np.float32)
    parity.check_fp32(first[0].cpu().numpy(), orc.gemm(A, B, one, 0, one, 0))


@pytest.mark.parametrize("M,N,K", [(16, 8192, 8192), (16, 4096, 4096), (1, 2048, 4096), (32, 1024, 8192),
                                   (40, 2048, 8192)])
def test_split_k_cluster_equals_global_bitwise(gb, orc, M, N, K):
    """A single call splits its tiles' K range across the CTAs of a cluster
    (partials added through distributed shared memory) when that fits; the
    same problem inside a grouped launch takes the global-memory split path.
    Both add the slices in the same order: bitwise equal, and within the
    tolerance of the oracle."""
    A = _codes(workloads.random_codes((M, K), seed=M + 21))
    B = _codes(workloads.random_codes((N, K), seed=N + 22))
    sa = torch.from_numpy(np.abs(workloads.randn_f32((M,), seed=5)) + 0.5).cuda()
    sb = torch.from_numpy(np.abs(workloads.randn_f32((N,), seed=6)) + 0.5).cuda()
    single = gb.gemm_fp8_dense(A, B, sa, 1, sb, 1, 1.0, gb.OUT_F32)
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    X = _codes(workloads.random_codes((64, 256), seed=3))
    Y = _codes(workloads.random_codes((64, 256), seed=4))
    one = _ones(64)
    Cx = torch.empty((64, 64), dtype=torch.float32, device="cuda")
    gb.gemm_fp8_grouped([gb.make_problem(A, B, sa, 1, sb, 1, C, 1.0, gb.OUT_F32),
                         gb.make_problem(X, Y, one, 1, one, 1, Cx, 1.0, gb.OUT_F32)])
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    assert torch.equal(single, C)
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    ref = orc.gemm(Ah, Bh, sa.cpu().numpy(), 1, sb.cpu().numpy(), 1)
    parity.check_fp32(single.cpu().numpy(), ref)


def test_split_k_integers_exact(gb, orc):
    A = workloads.small_int_codes((8, 6144), seed=91)
    B = workloads.small_int_codes((2048, 6144), seed=92)
    one = np.ones(1, np.float32)
    C = _gemm(gb, A, B, one, 0, one, 0, 1.0, gb.OUT_F32)
    assert np.array_equal(C.astype(np.float64), orc.gemm(A, B, one, 0, one, 0))


@pytest.mark.parametrize("M,N,K", [(16, 4096, 4096), (512, 1024, 2048)])
def test_dependent_chain_back_to_back_equals_synchronised(gb, M, N, K):
    """GEMMs launch with programmatic dependent launch (their setup may
    overlap the previous kernel) and wait for it before reading operands.
    A chain whose every step reads the previous step's output - quantise,
    GEMM, quantise that result, GEMM - enqueued back to back must give
    bitwise what the same steps give with a device sync after each."""
    dev = torch.device("cuda")
    x = torch.from_numpy(workloads.randn_f32((M, K), seed=M + 31)).to(dev)
    w1 = torch.from_numpy(workloads.randn_f32((N, K), seed=N + 32)).to(dev)
    w2 = torch.from_numpy(workloads.randn_f32((K, N), seed=K + 33)).to(dev)
    W1, d1 = gb.fp8_quantize_e4m3(w1, 1)
    W2, d2 = gb.fp8_quantize_e4m3(w2, 1)
    torch.cuda.synchronize()

    def chain(sync):
        q, dq = gb.fp8_quantize_e4m3(x, 1)
        if sync:
            torch.cuda.synchronize()
        h = gb.gemm_fp8_dense(q, W1, dq, 1, d1, 1, 1.0, gb.OUT_F32)
        if sync:
            torch.cuda.synchronize()
        qh, dh = gb.fp8_quantize_e4m3(h, 1)
        if sync:
            torch.cuda.synchronize()
        y = gb.gemm_fp8_dense(qh, W2, dh, 1, d2, 1, 1.0, gb.OUT_F32)
        torch.cuda.synchronize()
        return h, y

    h_ref, y_ref = chain(True)
    for _ in range(3):
        h, y = chain(False)
        assert torch.equal(h, h_ref) and torch.equal(y, y_ref)
    assert gb.fp8_last_device_error() == 0


def _int_values(shape, seed):
    """The integers behind workloads.small_int_codes(shape, seed) (same draw)."""
    return workloads.randint_f32(shape, seed, -4, 4).astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(128, 256, 262144), (16, 2048, 131072), (1, 4096, 131072),
                                   (1 << 20, 16, 128), (16, 1 << 20, 128), (3, 5, 262160)])
def test_extreme_shapes_small_integers_exact(gb, orc, M, N, K):
    """Very long K (split-K over many k-blocks; partial sums up to 4.2e6,
    still exact in FP32), a million-row M or N (8192 tiles; the swapped
    skinny path for N), and a ragged long K: every entry equals the integer
    product (float64 BLAS on the integers is exact below 2^53), and sampled
    entries equal the oracle's."""
    A = workloads.small_int_codes((M, K), seed=M + 11)
    B = workloads.small_int_codes((N, K), seed=N + 12)
    one = np.ones(1, np.float32)
    C = _gemm(gb, A, B, one, 0, one, 0, 1.0, gb.OUT_F32)
    exact = _int_values((M, K), M + 11) @ _int_values((N, K), N + 12).T
    assert np.array_equal(C.astype(np.float64), exact)
    ms, ns = workloads.sample_pairs(M, N, 256, seed=9)
    assert np.array_equal(C[ms, ns].astype(np.float64), orc.gemm_sampled(A, B, one, 0, one, 0, 1.0, ms, ns))


def test_grouped_long_list_equals_single_calls(gb, orc):
    """70 problems (more than one launch holds) give the bits of 70 single calls."""
    rng = np.random.default_rng(5)
    probs, outs, refs, keep = [], [], [], []
    for i in range(70):
        M, N, K = (int(v) for v in rng.integers(1, 9, 3) * 64)
        A, dA = orc.quantize(workloads.randn_f32((M, K), seed=2000 + i), 1)
        B, dB = orc.quantize(workloads.randn_f32((N, K), seed=3000 + i), 1)
        t = [_cuda(v) for v in (A, B, dA, dB)]
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        keep += t
        outs.append(C)
        probs.append(gb.make_problem(t[0], t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16))
        refs.append(gb.gemm_fp8_dense(t[0], t[1], t[2], 1, t[3], 1, 1.0, gb.OUT_BF16))
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    for a, b in zip(outs, refs):
        assert torch.equal(a, b)
