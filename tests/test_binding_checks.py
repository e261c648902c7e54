"""CPU checks of the Python binding's argument validation: arrays the
library writes or reads without a stride must have exactly the extent the
call uses, so that a wrong tensor is refused on the host instead of being
overrun on the device."""
import pytest
import torch

import paper_2602_10262_gb300 as gb


def test_shape_must_match_exactly():
    gb._shape(torch.empty(3, 4), "C", (3, 4))
    for shp in ((3, 3), (2, 4), (4, 4)):
        with pytest.raises(ValueError, match="C must have shape"):
            gb._shape(torch.empty(*shp), "C", (3, 4))


def test_packed_arrays_must_be_contiguous():
    gb._packed(torch.empty(4, 8), "a_vals")
    gb._packed(torch.empty(0, 8)[:, :4], "a_vals")          # empty: nothing to read
    with pytest.raises(ValueError, match="contiguous"):
        gb._packed(torch.empty(4, 8)[:, :4], "a_vals")


def test_scale_vectors_must_be_float32_on_the_gpu():
    for bad in (torch.ones(4), torch.ones(4, dtype=torch.float64), [1.0] * 4, None):
        with pytest.raises(TypeError, match="float32 CUDA tensor"):
            gb._scale(bad, "a_scale", 4)


def test_wrappers_refuse_host_tensors():
    x = torch.ones(4, 16)
    with pytest.raises(TypeError, match="CUDA tensor"):
        gb.fp8_quantize_e4m3(x, 1)
    with pytest.raises(TypeError, match="CUDA tensor"):
        gb.fp8_quantize_e5m2(x, 1)
    a = torch.zeros(4, 16, dtype=torch.uint8)
    with pytest.raises(TypeError, match="CUDA tensor"):
        gb.gemm_fp8_dense(a, a, torch.ones(1), 0, torch.ones(1), 0)
    with pytest.raises(TypeError, match="CUDA tensor"):
        gb.make_problem(a, a, torch.ones(1), 0, torch.ones(1), 0, torch.empty(4, 4))


def test_server_argument_checks():
    from paper_2602_10262_gb300 import server
    server._check_2d(0x1000, "x", torch.float32, 4, 16, 16)       # raw addresses pass unchecked
    with pytest.raises(TypeError, match="CUDA tensor"):
        server._check_2d(torch.ones(4, 16), "x", torch.float32, 4, 16, 16)
    with pytest.raises(TypeError, match="CUDA tensor"):
        server._check_weight(8, 16, torch.zeros(8, 16, dtype=torch.uint8), 16, None, 0x1000, 1)
