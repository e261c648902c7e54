"""GPU tests of the request server: results in the mix equal the same request
run alone (bitwise), in batched and per-call modes and with the bulk CTA cap,
and agree with the oracle."""
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


@pytest.fixture(scope="module")
def setup(gb):
    K = 512
    dev = torch.device("cuda")
    w_dense = torch.from_numpy(workloads.randn_f32((1024, K), seed=61)).to(dev)
    w_sparse = torch.from_numpy(workloads.randn_f32((768, K), seed=62)).to(dev)
    Wd, dWd = gb.fp8_quantize_e4m3(w_dense, 1)
    Ws, dWs = gb.fp8_quantize_e4m3(w_sparse, 1)
    vals, meta = gb.prune24_compress(Ws)
    Ms = [1, 7, 16, 64, 129, 300, 513, 2, 33, 200]
    xs = [torch.from_numpy(workloads.randn_f32((m, K), seed=100 + i)).to(dev) for i, m in enumerate(Ms)]
    torch.cuda.synchronize()
    return dict(K=K, Wd=Wd, dWd=dWd, vals=vals, meta=meta, dWs=dWs, Ms=Ms, xs=xs)


def _alone(gb, S, i, sparse):
    """The request computed by direct C-ABI calls (quantise, one GEMM)."""
    x = S["xs"][i]
    q, d = gb.fp8_quantize_e4m3(x, 1)
    if sparse:
        return gb.gemm_fp8_sparse24(S["vals"], S["meta"], q, S["dWs"], 1, d, 1, 1.0, gb.OUT_BF16,
                                    out_transposed=True)
    return gb.gemm_fp8_dense(q, S["Wd"], d, 1, S["dWd"], 1, 1.0, gb.OUT_BF16)


def _serve(gb, S, **cfg):
    from paper_2602_10262_gb300.server import Server
    outs, tickets = [], []
    with Server(num_tenants=2, latency_tenant=0, pool_bytes=256 << 20, **cfg) as srv:
        hd = srv.register_weight(1024, S["K"], S["Wd"], S["dWd"], 1)
        hs = srv.register_weight(768, S["K"], S["vals"], S["dWs"], 1, W_meta=S["meta"])
        for i, (m, x) in enumerate(zip(S["Ms"], S["xs"])):
            sparse = i % 2 == 1
            N = 768 if sparse else 1024
            out = torch.empty((m, N), dtype=torch.bfloat16, device="cuda")
            outs.append(out)
            tickets.append(srv.submit(i % 2, hs if sparse else hd, m, x, x.stride(0), out, N))
        res = [srv.wait(t, 30) for t in tickets]
        stats = srv.stats()
    assert all(r is not None and r.status == 0 for r in res)
    return outs, res, stats


@pytest.mark.parametrize("cfg", [dict(batching=True), dict(batching=False),
                                 dict(batching=True, bulk_max_ctas=40, max_batch=3)])
def test_mix_equals_alone_bitwise(gb, setup, cfg):
    outs, res, stats = _serve(gb, setup, **cfg)
    for i, out in enumerate(outs):
        ref = _alone(gb, setup, i, i % 2 == 1)
        assert torch.equal(out, ref), f"request {i} (M={setup['Ms'][i]})"
    assert stats["completed"] == len(outs)
    if cfg["batching"]:
        assert stats["kernel_launches"] < 2 * len(outs) or stats["batches"] == len(outs)
    else:
        assert stats["kernel_launches"] == 2 * len(outs)


@pytest.mark.parametrize("batching", [True, False])
def test_batch_intervals(gb, setup, batching):
    """Device start and end of each batch: start <= end; the batches of one
    tenant share a stream and do not overlap (1 us of clock-mapping slack);
    requests of one batch share the interval."""
    from paper_2602_10262_gb300.server import overlap_efficiency
    _, res, _ = _serve(gb, setup, batching=batching)
    for r in res:
        assert r.t_start_us <= r.t_end_us
    for t in (0, 1):
        spans = sorted({(r.t_start_us, r.t_end_us) for i, r in enumerate(res) if i % 2 == t})
        for (a0, b0), (a1, b1) in zip(spans, spans[1:]):
            assert a1 >= b0 - 1.0, (t, spans)
    assert 0.0 <= overlap_efficiency(res) <= 1.0


def test_server_results_vs_oracle(gb, orc, setup):
    outs, _, _ = _serve(gb, setup, batching=True)
    Wd = setup["Wd"].cpu().numpy()
    dWd = setup["dWd"].cpu().numpy()
    vals, meta = setup["vals"].cpu().numpy(), setup["meta"].cpu().numpy()
    dWs = setup["dWs"].cpu().numpy()
    K = setup["K"]
    for i in (0, 1, 4, 5):
        x = setup["xs"][i].cpu().numpy()
        q, d = orc.quantize(x, 1)
        if i % 2:
            ref = orc.gemm_sparse24(vals, meta, q, K, dWs, 1, d, 1).T
            S = orc.gemm_sparse24(parity.abs_codes(vals), meta, parity.abs_codes(q), K, dWs, 1, d, 1).T
        else:
            ref = orc.gemm(q, Wd, d, 1, dWd, 1)
            S = orc.gemm(parity.abs_codes(q), parity.abs_codes(Wd), d, 1, dWd, 1)
        parity.check_bf16(outs[i].float().cpu().numpy(), ref, S, K)


def test_server_pool_from_free_memory(gb):
    from paper_2602_10262_gb300.server import Server
    free, _ = torch.cuda.mem_get_info()
    reserve = max(free - (512 << 20), 1 << 20)     # leave the pool ~512 MiB
    with Server(num_tenants=1, latency_tenant=-1, reserve_bytes=reserve) as srv:
        st = srv.stats()
        assert 0 < st["pool_bytes"] <= free - reserve + (1 << 20)


@pytest.fixture(scope="module")
def setup_e5m2(gb, setup):
    """The same requests against E5M2 weights (dense and 2:4)."""
    K = setup["K"]
    dev = torch.device("cuda")
    w_dense = torch.from_numpy(workloads.randn_f32((1024, K), seed=61)).to(dev)
    w_sparse = torch.from_numpy(workloads.randn_f32((768, K), seed=62)).to(dev)
    Wd, dWd = gb.fp8_quantize_e5m2(w_dense, 1)
    Ws, dWs = gb.fp8_quantize_e5m2(w_sparse, 1)
    vals, meta = gb.prune24_compress(Ws)
    torch.cuda.synchronize()
    return dict(setup, Wd=Wd, dWd=dWd, vals=vals, meta=meta, dWs=dWs)


@pytest.mark.parametrize("batching", [True, False])
def test_e5m2_weights_equal_direct_calls_bitwise(gb, orc, setup_e5m2, batching):
    """Requests against E5M2 weights (E4M3 activations x E5M2 weights, the
    FP8 x BF8 pairing) equal direct format-aware calls bit for bit, and a
    dense one matches the oracle."""
    from paper_2602_10262_gb300.server import Server
    S = setup_e5m2
    outs, tickets = [], []
    with Server(num_tenants=2, latency_tenant=0, batching=batching, pool_bytes=256 << 20) as srv:
        hd = srv.register_weight(1024, S["K"], S["Wd"], S["dWd"], 1, w_format=1)
        hs = srv.register_weight(768, S["K"], S["vals"], S["dWs"], 1, W_meta=S["meta"], w_format=1)
        for i, (m, x) in enumerate(zip(S["Ms"], S["xs"])):
            sparse = i % 2 == 1
            N = 768 if sparse else 1024
            out = torch.empty((m, N), dtype=torch.bfloat16, device="cuda")
            outs.append(out)
            tickets.append(srv.submit(i % 2, hs if sparse else hd, m, x, x.stride(0), out, N))
        res = [srv.wait(t, 30) for t in tickets]
    assert all(r is not None and r.status == 0 for r in res)
    for i, out in enumerate(outs):
        q, d = gb.fp8_quantize_e4m3(S["xs"][i], 1)
        if i % 2:
            ref = gb.gemm_fp8_sparse24_fmt(S["vals"], S["meta"], q, S["dWs"], 1, d, 1, 1.0, gb.OUT_BF16,
                                           True, gb.E5M2, gb.E4M3)
        else:
            ref = gb.gemm_fp8_dense_fmt(q, S["Wd"], d, 1, S["dWd"], 1, 1.0, gb.OUT_BF16, gb.E4M3, gb.E5M2)
        assert torch.equal(out, ref), f"request {i}"
    x = S["xs"][4].cpu().numpy()
    qo, do = orc.quantize(x, 1)
    Wd, dWd = S["Wd"].cpu().numpy(), S["dWd"].cpu().numpy()
    ref = orc.gemm(qo, Wd, do, 1, dWd, 1, a_fmt=0, b_fmt=1)
    Sm = orc.gemm(parity.abs_codes(qo), parity.abs_codes(Wd), do, 1, dWd, 1, a_fmt=0, b_fmt=1)
    parity.check_bf16(outs[4].float().cpu().numpy(), ref, Sm, S["K"])
