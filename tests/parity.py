"""Tolerances and comparison helpers shared by the GPU parity tests.

FP32 output: normwise relative error ||C - C_ref||_F / ||C_ref||_F <= 1e-5
against the FP64 oracle on the same decoded inputs.

BF16 output: per element |C - C_ref| <= 1e-2 * |C_ref| + gamma * S, where
S = |alpha * dA[m] * dB[n]| * sum_k |dec(A[m,k]) dec(B[n,k])| and
gamma = (K + 2) * 2^-24.  The first term is the stated 1e-2 relative bound
(bf16 rounding alone is <= 2^-9); the second is the standard componentwise
bound for a K-term FP32-accumulated dot product plus the two FP32 scale
multiplies, and only matters where C_ref cancels to near zero.  Tests
report how many elements needed the second term.
"""
from __future__ import annotations

import numpy as np

FP32_NORMWISE = 1e-5
BF16_REL = 1e-2


def abs_codes(c: np.ndarray) -> np.ndarray:
    """Codes of |value| (clear the sign bit)."""
    return c & np.uint8(0x7F)


def check_fp32(C: np.ndarray, ref: np.ndarray):
    C = C.astype(np.float64)
    num = np.linalg.norm(C - ref)
    den = np.linalg.norm(ref)
    err = num / den if den > 0 else num
    assert err <= FP32_NORMWISE, f"normwise relative error {err:.3e} > {FP32_NORMWISE}"
    return err


def check_bf16(C: np.ndarray, ref: np.ndarray, S: np.ndarray, K: int):
    C = C.astype(np.float64)
    gamma = (K + 2) * 2.0 ** -24
    diff = np.abs(C - ref)
    rel_ok = diff <= BF16_REL * np.abs(ref)
    ok = rel_ok | (diff <= BF16_REL * np.abs(ref) + gamma * S)
    bad = np.count_nonzero(~ok)
    if bad:
        idx = np.argwhere(~ok)[0]
        raise AssertionError(
            f"{bad} elements outside tolerance; first at {tuple(idx)}: got {C[tuple(idx)]}, "
            f"ref {ref[tuple(idx)]}, S {S[tuple(idx)]}")
    return int(np.count_nonzero(~rel_ok))
