"""Pins for the oracle's GEMM C = alpha * dA[m] * dB[n] * sum_k dec(A) dec(B)
(the FP8 x FP8 -> wide-accumulation matrix operation of paper section 4).

Checked against: numpy float64 matmul on inputs decoded by PyTorch's
float8_e4m3fn cast (library routines), exact rational sums (brute force with
fractions on tiny cases), the identity, permutation invariants, and sparse =
dense on the decompressed pruned matrix (section 6).
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import workloads


def _torch_dec(codes):
    return torch.from_numpy(np.ascontiguousarray(codes)).view(torch.float8_e4m3fn).to(torch.float64).numpy()


@pytest.mark.parametrize("a_mode,b_mode", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (3, 5, 7), (17, 9, 64), (40, 33, 200)])
def test_vs_numpy_matmul(orc, M, N, K, a_mode, b_mode):
    A = workloads.random_codes((M, K), seed=M + 100)
    B = workloads.random_codes((N, K), seed=N + 200)
    dA = np.abs(workloads.randn_f32((M,), seed=3)) + 0.5
    dB = np.abs(workloads.randn_f32((N,), seed=4)) + 0.5
    alpha = 0.75
    C = orc.gemm(A, B, dA, a_mode, dB, b_mode, alpha)
    sa = dA.astype(np.float64) if a_mode else np.full(M, float(dA[0]))
    sb = dB.astype(np.float64) if b_mode else np.full(N, float(dB[0]))
    ref = alpha * sa[:, None] * sb[None, :] * (_torch_dec(A) @ _torch_dec(B).T)
    assert C.shape == (M, N)
    np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_exact_rational_sum(orc):
    A = workloads.random_codes((1, 40), seed=21)
    B = workloads.random_codes((1, 40), seed=22)
    da, db = _torch_dec(A)[0], _torch_dec(B)[0]
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(da, db))
    C = orc.gemm(A, B, np.ones(1, np.float32), 0, np.ones(1, np.float32), 0)
    assert abs(Fraction(C[0, 0]) - exact) <= abs(exact) * Fraction(1, 2 ** 50) + Fraction(1, 2 ** 100)


def test_small_integers_exact(orc):
    A = workloads.small_int_codes((16, 300), seed=23)
    B = workloads.small_int_codes((12, 300), seed=24)
    C = orc.gemm(A, B, np.ones(1, np.float32), 0, np.ones(1, np.float32), 0)
    ia = _torch_dec(A).astype(np.int64)
    ib = _torch_dec(B).astype(np.int64)
    assert np.array_equal(C, (ia @ ib.T).astype(np.float64))


def test_identity(orc):
    K = 48
    A = workloads.random_codes((10, K), seed=25)
    one = torch.tensor([1.0]).to(torch.float8_e4m3fn).view(torch.uint8).item()
    I = np.zeros((K, K), np.uint8)
    I[np.arange(K), np.arange(K)] = one
    C = orc.gemm(A, I, np.ones(1, np.float32), 0, np.ones(1, np.float32), 0)
    assert np.array_equal(C, _torch_dec(A))


def test_permutations(orc):
    A = workloads.random_codes((20, 64), seed=26)
    B = workloads.random_codes((15, 64), seed=27)
    dA = np.abs(workloads.randn_f32((20,), seed=28)) + 0.1
    dB = np.abs(workloads.randn_f32((15,), seed=29)) + 0.1
    C = orc.gemm(A, B, dA, 1, dB, 1)
    p = np.random.default_rng(0).permutation(20)
    assert np.array_equal(orc.gemm(A[p], B, dA[p], 1, dB, 1), C[p])
    q = np.random.default_rng(1).permutation(15)
    assert np.array_equal(orc.gemm(A, B[q], dA, 1, dB[q], 1), C[:, q])
    k = np.random.default_rng(2).permutation(64)
    np.testing.assert_allclose(orc.gemm(A[:, k], B[:, k], dA, 1, dB, 1), C, rtol=1e-12,
                               atol=1e-12 * np.abs(C).max())


def test_sampled_equals_full(orc):
    A = workloads.random_codes((50, 96), seed=30)
    B = workloads.random_codes((40, 96), seed=31)
    dA = np.abs(workloads.randn_f32((50,), seed=32)) + 0.1
    dB = np.abs(workloads.randn_f32((40,), seed=33)) + 0.1
    C = orc.gemm(A, B, dA, 1, dB, 1, 2.0)
    ms, ns = workloads.sample_pairs(50, 40, 500, seed=34)
    assert np.array_equal(orc.gemm_sampled(A, B, dA, 1, dB, 1, 2.0, ms, ns), C[ms, ns])


def test_sparse_equals_dense_on_pruned(orc):
    A = workloads.random_codes((24, 128), seed=35)
    B = workloads.random_codes((20, 128), seed=36)
    dA = np.abs(workloads.randn_f32((24,), seed=37)) + 0.1
    dB = np.abs(workloads.randn_f32((20,), seed=38)) + 0.1
    v, m = orc.prune24(A)
    Ap = orc.decompress24(v, m, 128)
    Cs = orc.gemm_sparse24(v, m, B, 128, dA, 1, dB, 1, 1.5)
    Cd = orc.gemm(Ap, B, dA, 1, dB, 1, 1.5)
    assert np.array_equal(Cs, Cd)
    # and the pruning really dropped terms: the unpruned product differs
    assert not np.allclose(Cd, orc.gemm(A, B, dA, 1, dB, 1, 1.5))
