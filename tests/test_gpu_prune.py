"""GPU parity: prune24_compress / prune24_decompress against the oracle,
bit-exact on kept codes and metadata."""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


def _ties(a):
    a = a.copy()
    a[:, 1::5] = a[:, 0::5][:, : a[:, 1::5].shape[1]]      # equal neighbours
    a[:, 2::9] ^= 0x80                                       # equal magnitude, other sign
    return a


@pytest.mark.parametrize("shape", [(1, 4), (3, 36), (5, 48), (7, 1028), (33, 1040), (128, 256),
                                   (257, 4096), (64, 100), (2, 16)])
def test_parity(gb, orc, shape):
    a = _ties(workloads.random_codes(shape, seed=shape[1]))
    v, m = gb.prune24_compress(torch.from_numpy(a).cuda())
    vo, mo = orc.prune24(a)
    assert np.array_equal(v.cpu().numpy(), vo)
    assert np.array_equal(m.cpu().numpy(), mo)


def test_parity_full_size(gb, orc):
    x = workloads.randn_f32((8192, 8192), seed=workloads.SEED_A)
    q, _ = orc.quantize(x, 1)
    v, m = gb.prune24_compress(torch.from_numpy(q).cuda())
    vo, mo = orc.prune24(q)
    assert np.array_equal(m.cpu().numpy(), mo)
    assert np.array_equal(v.cpu().numpy(), vo)


def test_strided_input(gb, orc):
    wide = workloads.random_codes((50, 300), seed=9)
    at = torch.from_numpy(wide).cuda()[:, 4:260]            # lda = 300, K = 256
    v, m = gb.prune24_compress(at)
    vo, mo = orc.prune24(wide[:, 4:260])
    assert np.array_equal(v.cpu().numpy(), vo) and np.array_equal(m.cpu().numpy(), mo)


def test_decompress(gb, orc):
    a = _ties(workloads.random_codes((33, 512), seed=10))
    v, m = gb.prune24_compress(torch.from_numpy(a).cuda())
    d = gb.prune24_decompress(v, m, 512)
    assert np.array_equal(d.cpu().numpy(), orc.decompress24(*orc.prune24(a), 512))


def test_bad_k(gb):
    with pytest.raises(gb.Fp8Error) as e:
        gb.prune24_compress(torch.zeros((2, 6), dtype=torch.uint8, device="cuda"))
    assert e.value.status == -2
