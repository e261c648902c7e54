"""Sampled oracle checks for products too large for the full FP64 oracle.

Each entry of C is an independent dot product, so a seeded sample of
entries (plus whole rows and columns) checks the product at any size.  Per-row
scale selection is row-local, so the oracle quantises (and, for 2:4 operands,
prunes) only the rows of A and B that the sample touches, from the same fp32
inputs the GPU path started from: no oracle input comes from the CUDA path.
"""
from __future__ import annotations

import numpy as np

import workloads
from tests import parity


def entries(M: int, N: int, n: int = 4096, seed: int = 99, lines: bool = True):
    """n seeded (m, n) pairs, plus (with lines) the first and last rows and
    the first and last columns in full."""
    ms, ns = workloads.sample_pairs(M, N, n, seed=seed)
    if lines:
        rows = np.array([0, M - 1])
        cols = np.array([0, N - 1])
        ms = np.concatenate([ms, np.repeat(rows, N), np.tile(np.arange(M), 2)])
        ns = np.concatenate([ns, np.tile(np.arange(N), 2), np.repeat(cols, M)])
    return ms, ns


def reference(orc, x, w, ms, ns, alpha=1.0, sparse_w=False, fmt_w=0):
    """Oracle values and the bound's S term at (ms, ns) of
    C = alpha * dX dW dec(q(x)) dec(q(w))^T, x [M, K] and w [N, K] fp32,
    both quantised per row by the oracle (x to E4M3, w to fmt_w); with
    sparse_w the quantised w is 2:4-pruned first."""
    ua, ia = np.unique(ms, return_inverse=True)
    ub, ib = np.unique(ns, return_inverse=True)
    A, dA = orc.quantize(np.ascontiguousarray(x[ua]), 1)
    B, dB = orc.quantize(np.ascontiguousarray(w[ub]), 1, fmt=fmt_w)
    if sparse_w:
        K = B.shape[1]
        vals, meta = orc.prune24(B)
        B = orc.decompress24(vals, meta, K)
    ref = orc.gemm_sampled(A, B, dA, 1, dB, 1, alpha, ia, ib, a_fmt=0, b_fmt=fmt_w)
    S = orc.gemm_sampled(parity.abs_codes(A), parity.abs_codes(B), dA, 1, dB, 1, abs(alpha), ia, ib,
                         a_fmt=0, b_fmt=fmt_w)
    return ref, S
