"""GPU tests of the autotuner (tile cache) and of the CUDA-graph grouped
launch: both change how the work is launched, never the results."""
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


def _problems(gb, orc, shapes, seed):
    probs, outs, keep = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        x = workloads.randn_f32((M, K), seed=seed + 2 * i)
        w = workloads.randn_f32((N, K), seed=seed + 2 * i + 1)
        A, dA = orc.quantize(x, 1)
        B, dB = orc.quantize(w, 1)
        t = [torch.from_numpy(v).cuda() for v in (A, B, dA, dB)]
        C = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
        keep += t
        outs.append(C)
        probs.append(gb.make_problem(t[0], t[1], t[2], 1, t[3], 1, C, 1.0, gb.OUT_BF16))
    return probs, outs, keep


SHAPES = [(1024, 768, 1024), (512, 2048, 512), (2048, 1024, 256), (16, 4096, 2048)]


def test_autotune_picks_a_config_and_keeps_results(gb, orc, tmp_path):
    probs, outs, keep = _problems(gb, orc, SHAPES, 500)
    gb.gemm_fp8_tune_cache_clear()
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    before = [c.clone() for c in outs]
    best = gb.gemm_fp8_grouped_autotune(probs, iters=2)
    assert best["mt"] in (1, 2, 3) and best["group_m"] in (2, 4, 8, 16, 32)
    assert best["bn_max"] in (0, 64, 128)
    assert best["ms_per_launch"] > 0
    for c in outs:
        c.zero_()
    gb.gemm_fp8_grouped(probs)             # uses the cached choice
    torch.cuda.synchronize()
    for a, b in zip(before, outs):
        assert torch.equal(a, b)
    path = str(tmp_path / "tiles.txt")
    gb.gemm_fp8_tune_cache_save(path)
    text = open(path).read()
    assert f" {best['mt']} {best['group_m']} {best['bn_max']}\n" in text
    gb.gemm_fp8_tune_cache_clear()
    gb.gemm_fp8_tune_cache_load(path)
    assert gb.fp8_last_device_error() == 0
    gb.gemm_fp8_tune_cache_clear()


def test_graph_launch_equals_direct_and_updates_pointers(gb, orc):
    probs1, outs1, keep1 = _problems(gb, orc, SHAPES, 600)
    probs2, outs2, keep2 = _problems(gb, orc, SHAPES, 700)
    gb.gemm_fp8_grouped(probs1)
    gb.gemm_fp8_grouped(probs2)
    torch.cuda.synchronize()
    ref1 = [c.clone() for c in outs1]
    ref2 = [c.clone() for c in outs2]
    for c in outs1 + outs2:
        c.zero_()
    g = gb.GroupedGraph(probs1)
    for _ in range(2):                     # replays reuse the graph's split-K workspace
        for c in outs1:
            c.zero_()
        g.launch()
        torch.cuda.synchronize()
        for a, b in zip(ref1, outs1):
            assert torch.equal(a, b)
    g.update(probs2)                       # same shapes, new pointers: no re-capture
    g.launch()
    torch.cuda.synchronize()
    for a, b in zip(ref2, outs2):
        assert torch.equal(a, b)
    probs3, _, keep3 = _problems(gb, orc, [(1024, 768, 512)] + SHAPES[1:], 800)
    with pytest.raises(gb.Fp8Error) as e:
        g.update(probs3)
    assert e.value.status == -2
    g.close()
    assert gb.fp8_last_device_error() == 0
