"""Width and rounding of the tensor-core FP32 accumulation, measured.

Each output entry is C = 2^16 + b: one large product (256 x 256, at k = 0)
and one small product b (1 x b) placed in the same 32-wide K step as the
large one (k = 1, the same MMA instruction), in a later MMA of the same
128-wide k-block (k = 64), in the next k-block (k = 128, a later MMA adding
into the accumulator), or before the large product (small at k = 0, large at
k = 128).  b runs over E4M3 values from 2^-1 down to 2^-9, i.e. from 2^6 ulp
down to 1/4 ulp of 2^16 in FP32 (ulp 2^-7), including the half-ulp tie
2^-8 and 3/4 ulp.  All scales are 1 and the output is FP32, so the stored
value is the accumulator itself.

An accumulator with a 24-bit significand that rounds to nearest gives
fl32(2^16 + b) rounded to nearest even; one that truncates gives it rounded
toward zero.  The test requires every result to be one of those two roundings
of the exact sum (the accumulator holds at least FP32's 24 bits, unit
roundoff <= 2^-23), and prints which one each placement shows.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SMALL = [2.0 ** -1, 2.0 ** -2, 2.0 ** -3, 2.0 ** -4, 2.0 ** -5, 2.0 ** -6, 1.75 * 2.0 ** -7,
         1.5 * 2.0 ** -7, 1.25 * 2.0 ** -7, 2.0 ** -7, 1.5 * 2.0 ** -8, 2.0 ** -8, 2.0 ** -9]
# (k of the large product, k of the small one)
PLACEMENTS = {"same MMA (k=1)": (0, 1), "same k-block (k=64)": (0, 64),
              "next k-block (k=128)": (0, 128), "small first (k=0, large k=128)": (128, 0)}
K = 256


def _code(v):
    c = torch.tensor([v], dtype=torch.float32).to(torch.float8_e4m3fn)
    assert float(c.float()) == v, v                  # exactly representable
    return int(c.view(torch.uint8))


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


def test_accumulator_keeps_fp32_width(gb):
    names = list(PLACEMENTS)
    N = len(SMALL)
    # placement r: rows [32 r, 32 r + 32) of A and columns [N r, N r + N) of
    # B; only that diagonal block of C is read, C = 256 * 256 + 1 * b_n
    A = np.zeros((32 * len(names), K), np.uint8)
    B = np.zeros((N * len(names), K), np.uint8)
    big, one = _code(256.0), _code(1.0)
    for r, name in enumerate(names):
        kb, ks = PLACEMENTS[name]
        A[32 * r:32 * r + 32, kb] = big
        A[32 * r:32 * r + 32, ks] = one
        for n, b in enumerate(SMALL):
            B[N * r + n, kb] = big
            B[N * r + n, ks] = _code(b)

    dev = torch.device("cuda")
    At, Bt = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    one_s = torch.ones(1, device=dev)
    C = gb.gemm_fp8_dense(At, Bt, one_s, 0, one_s, 0, 1.0, gb.OUT_F32)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    C = C.cpu().numpy()

    bad = []
    for r, name in enumerate(names):
        blk = C[32 * r:32 * r + 32, N * r:N * r + N]
        assert (blk == blk[0]).all(), f"{name}: rows of one placement differ"
        print(f"\n{name}:")
        for n, b in enumerate(SMALL):
            got = float(blk[0, n])
            exact = 65536.0 + b
            rne = float(np.float32(65536.0) + np.float32(b))      # numpy rounds to nearest even
            rz = rne if rne <= exact else float(np.nextafter(np.float32(rne), np.float32(0.0)))
            kind = ("exact" if got == exact else "nearest-even" if got == rne else
                    "toward-zero" if got == rz else "neither")
            print(f"  b = {b:.10g}: C - 2^16 = {got - 65536.0:.10g} ({kind})")
            if got not in (rne, rz):
                bad.append((name, b, got, exact))
    assert not bad, f"results outside both FP32 roundings of the exact sum: {bad}"
