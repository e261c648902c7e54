"""Seeded synthetic inputs and workload shapes for the FP8 GEMM path.

Shared by the tests, the smoke check and the benchmark.  This module holds no
arithmetic of the method (no quantisation, pruning, encoding or products): it
only draws random numbers from fixed seeds and names the shapes.

Recipe (the paper's microbenchmarks run on synthetic matrices; there is no
dataset): fp32 values drawn N(0, 1) from ``torch.Generator().manual_seed``
on the CPU, so the CPU oracle and the GPU see identical bits.  Seeds: 0 for A,
1 for B, 2 and up for serving requests.
"""
from __future__ import annotations

import numpy as np
import torch

SEED_A = 0
SEED_B = 1
SEED_REQUESTS = 2


def randn_f32(shape, seed: int) -> np.ndarray:
    """fp32 N(0,1) values, reproducible from ``seed`` on any machine."""
    g = torch.Generator().manual_seed(int(seed))
    return torch.randn(*shape, generator=g, dtype=torch.float32).numpy()


def randint_f32(shape, seed: int, lo: int, hi: int) -> np.ndarray:
    """fp32 integers uniform in [lo, hi]."""
    g = torch.Generator().manual_seed(int(seed))
    return torch.randint(lo, hi + 1, tuple(shape), generator=g).to(torch.float32).numpy()


def small_int_codes(shape, seed: int, maxabs: int = 4, fmt: int = 0) -> np.ndarray:
    """FP8 codes (fmt 0: E4M3, 1: E5M2) of integers uniform in [-maxabs, maxabs].

    The codes come from PyTorch's own float8_e4m3fn / float8_e5m2 cast (exact
    for integers up to 8 in both), so neither the oracle nor the CUDA path
    produces them.  With such inputs every partial sum of a GEMM is an integer
    far below 2^24, so an FP32-accumulated product is exact."""
    if fmt == 1 and maxabs > 8:
        raise ValueError("E5M2 holds the integers up to 8 exactly")
    v = torch.from_numpy(randint_f32(shape, seed, -maxabs, maxabs))
    dt = torch.float8_e5m2 if fmt == 1 else torch.float8_e4m3fn
    return v.to(dt).view(torch.uint8).numpy().copy()


def random_codes(shape, seed: int, fmt: int = 0) -> np.ndarray:
    """Uniform random finite FP8 codes.  fmt 0 (E4M3): every byte except 0x7F
    and 0xFF; fmt 1 (E5M2): every byte except 0x7C..0x7F and 0xFC..0xFF."""
    g = torch.Generator().manual_seed(int(seed))
    if fmt == 1:
        c = torch.randint(0, 248, tuple(shape), generator=g, dtype=torch.int32)
        c = torch.where(c >= 124, c + 4, c)       # skip 0x7C..0x7F
        return c.to(torch.uint8).numpy().copy()
    c = torch.randint(0, 254, tuple(shape), generator=g, dtype=torch.int32)
    c = torch.where(c >= 0x7F, c + 1, c)          # skip 0x7F
    return c.to(torch.uint8).numpy().copy()


def sample_pairs(M: int, N: int, n: int, seed: int):
    """Seeded (m, n) index pairs for sampled checks of large products."""
    g = torch.Generator().manual_seed(int(seed))
    ms = torch.randint(0, M, (n,), generator=g).numpy().astype(np.int64)
    ns = torch.randint(0, N, (n,), generator=g).numpy().astype(np.int64)
    return ms, ns


# Workload shapes (paper section 4 sweeps square and skinny FP8 GEMMs; section 6
# sweeps 2:4-sparse GEMMs against dense on the same operands; section 7.1 is a
# transformer-style sequence of GEMMs).
DENSE_SMALL = (256, 256, 256)
SQUARE_SWEEP = (1024, 2048, 4096, 8192, 16384)
SKINNY_M = (16, 64, 128)
SKINNY_NK = 8192
SPARSE_SQUARE = (2048, 4096, 8192, 16384)
SPARSE_SKINNY = (128, 8192, 8192)
SPARSE_RECT = (512, 2048, 1024)          # M x N x K the paper singles out in section 6
TOKENS = 8 * 2048
D_MODEL = 4096
TRANSFORMER_LAYER = (                    # (name, M, N, K): activations [M, K], weights [N, K]
    ("qkv", TOKENS, 12288, 4096),
    ("out", TOKENS, 4096, 4096),
    ("ffn_up", TOKENS, 14336, 4096),
    ("ffn_down", TOKENS, 4096, 14336),
)
