"""Pins for the oracle's 2:4 pruning / compression (paper section 2
"Structured Sparsity", section 6: two of every four consecutive elements
along K are zero).

Checked against: hand-built groups (tests/golden), a per-group Python
restatement by sorting, and invariants (exactly two kept, kept magnitudes
>= dropped, round trip through decompression).
"""
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _groups():
    rows = []
    with open(os.path.join(GOLDEN, "prune24_groups.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            codes, kept, vals, nib = [p.split() for p in line.split("|")]
            rows.append(([int(c, 16) for c in codes], [int(k) for k in kept],
                         [int(v, 16) for v in vals], int(nib[0], 16)))
    return rows


def test_golden_groups(orc):
    rows = _groups()
    assert len(rows) == 10
    for codes, kept, vals, nib in rows:
        v, m = orc.prune24(np.array([codes], np.uint8))
        assert list(v[0]) == vals, codes
        assert m[0, 0] == nib, codes
        assert (m[0, 0] & 3, m[0, 0] >> 2) == tuple(kept)


def test_golden_groups_packed_in_rows(orc):
    # the same groups laid out along one row: nibble g sits in byte g // 2,
    # low nibble for even g
    rows = _groups()
    a = np.array([sum((r[0] for r in rows), [])], np.uint8)
    v, m = orc.prune24(a)
    assert m.shape == (1, (len(rows) * 4 + 7) // 8)
    for g, (_, _, vals, nib) in enumerate(rows):
        assert list(v[0, 2 * g:2 * g + 2]) == vals
        assert (m[0, g // 2] >> (4 * (g % 2))) & 0xF == nib


def _restated(a):
    M, K = a.shape
    out = np.zeros_like(a)
    for r in range(M):
        for g in range(K // 4):
            grp = [int(c) for c in a[r, 4 * g:4 * g + 4]]
            order = sorted(range(4), key=lambda i: (-(grp[i] & 0x7F), i))
            for i in order[:2]:
                out[r, 4 * g + i] = grp[i]
    return out


@pytest.mark.parametrize("shape", [(1, 4), (5, 12), (32, 64), (7, 1028)])
def test_matches_sort_restatement(orc, shape):
    a = workloads.random_codes(shape, seed=shape[1])
    # plant ties: copy some elements onto their neighbours
    a[:, 1::7] = a[:, 0::7][:, : a[:, 1::7].shape[1]]
    v, m = orc.prune24(a)
    assert np.array_equal(orc.decompress24(v, m, shape[1]), _restated(a))


def test_invariants(orc):
    a = workloads.random_codes((64, 256), seed=11)
    v, m = orc.prune24(a)
    M, K = a.shape
    for g in range(K // 4):
        nib = (m[:, g // 2] >> (4 * (g % 2))) & 0xF
        i0, i1 = nib & 3, nib >> 2
        assert np.all(i0 < i1)
        grp = a[:, 4 * g:4 * g + 4]
        kept = np.stack([grp[np.arange(M), i0], grp[np.arange(M), i1]], 1)
        assert np.array_equal(kept, v[:, 2 * g:2 * g + 2])
        keys = grp & 0x7F
        mask = np.ones((M, 4), bool)
        mask[np.arange(M), i0] = False
        mask[np.arange(M), i1] = False
        dropped_max = np.where(mask, keys, 0).max(1)
        assert np.all(np.minimum(keys[np.arange(M), i0], keys[np.arange(M), i1]) >= dropped_max)


def test_roundtrip_on_pruned(orc):
    a = workloads.random_codes((16, 128), seed=12)
    v, m = orc.prune24(a)
    ap = orc.decompress24(v, m, 128)
    v2, m2 = orc.prune24(ap)
    assert np.array_equal(v, v2) and np.array_equal(m, m2)
    # each group of the pruned matrix has at most two nonzero codes
    nz = (ap.reshape(16, 32, 4) & 0x7F) != 0
    assert np.all(nz.sum(-1) <= 2)


def test_quantise_then_prune_keeps_amax(orc):
    x = workloads.randn_f32((8, 64), seed=13)
    q, d = orc.quantize(x, 1)
    v, _ = orc.prune24(q)
    assert np.all((v & 0x7F).max(1) == 0x7E)


def test_bad_k(orc):
    with pytest.raises(oracle.OracleError):
        orc.prune24(np.zeros((2, 6), np.uint8))
