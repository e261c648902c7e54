"""GPU parity at the full sizes of the transformer-layer and serving workloads.

- Transformer layer (paper section 7.1's sequence of FP8 GEMMs): tokens
  8 x 2048 = 16384, d_model 4096; QKV 4096 -> 12288, output 4096 -> 4096,
  FFN 4096 -> 14336 -> 4096, as four independent problems of one grouped
  persistent launch and as a replay of its CUDA graph.  Inputs start as fp32
  N(0, 1) and are quantised on the GPU (activations per row, weights per
  output channel, E4M3); outputs BF16.
- Serving mix (paper sections 5 and 6.2, the concurrent-GEMM question):
  requests with M log-uniform in [1, 4096] (tenant 0 small M, tenant 1
  large M), (N, K) uniform over {4096, 8192, 14336}^2, half of them on the
  2:4-pruned copy of the weight, served by the request server with
  continuous batching; every response is checked.

Each output is checked against the FP64 oracle on 4096 seeded entries plus
two full rows and two full columns (serving: 256 entries per response), with
the BF16 tolerance of tests/parity.py; the oracle quantises the sampled rows
itself from the same fp32 inputs.
"""
import numpy as np
import pytest
import torch

import workloads
from tests import parity, sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2602_10262_gb300 as gb
    gb.library()
    return gb


def _inputs(i, M, N, K):
    return (workloads.randn_f32((M, K), seed=40 + 2 * i),
            workloads.randn_f32((N, K), seed=41 + 2 * i))


@pytest.fixture(scope="module")
def layer(gb):
    """The four layer GEMMs quantised on the GPU, as grouped problems."""
    dev = torch.device("cuda")
    probs, outs, keep = [], [], []
    for i, (_, M, N, K) in enumerate(workloads.TRANSFORMER_LAYER):
        x, w = _inputs(i, M, N, K)
        xd, wd = torch.from_numpy(x).to(dev), torch.from_numpy(w).to(dev)
        A, dA = gb.fp8_quantize_e4m3(xd, 1)
        B, dB = gb.fp8_quantize_e4m3(wd, 1)
        del xd, wd
        C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
        keep += [A, dA, B, dB]
        outs.append(C)
        probs.append(gb.make_problem(A, B, dA, 1, dB, 1, C, 1.0, gb.OUT_BF16))
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    return probs, outs, keep


@pytest.fixture(scope="module")
def layer_refs(orc):
    refs = []
    for i, (_, M, N, K) in enumerate(workloads.TRANSFORMER_LAYER):
        x, w = _inputs(i, M, N, K)
        ms, ns = sampled.entries(M, N, seed=300 + i)
        ref, S = sampled.reference(orc, x, w, ms, ns)
        refs.append((ms, ns, ref, S, K))
    return refs


def _check_layer(outs, refs):
    for C, (ms, ns, ref, S, K) in zip(outs, refs):
        got = C[torch.from_numpy(ms).cuda(), torch.from_numpy(ns).cuda()].float().cpu().numpy()
        parity.check_bf16(got, ref, S, K)


def test_transformer_layer_grouped_sampled(gb, layer, layer_refs):
    probs, outs, _ = layer
    for C in outs:
        C.fill_(float("nan"))
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    assert gb.fp8_last_device_error() == 0
    _check_layer(outs, layer_refs)


def test_transformer_layer_graph_sampled(gb, layer, layer_refs):
    probs, outs, _ = layer
    gb.gemm_fp8_grouped(probs)
    torch.cuda.synchronize()
    direct = [C.clone() for C in outs]
    g = gb.GroupedGraph(probs)
    try:
        for _ in range(2):
            for C in outs:
                C.fill_(float("nan"))
            g.launch()
            torch.cuda.synchronize()
            for a, b in zip(direct, outs):
                assert torch.equal(a, b)
    finally:
        g.close()
    assert gb.fp8_last_device_error() == 0
    _check_layer(outs, layer_refs)


# ---------------------------------------------------------------- serving mix

SIZES = (4096, 8192, 14336)


def _trace(n):
    """Seeded requests: (tenant, M, N, K, sparse)."""
    g = torch.Generator().manual_seed(workloads.SEED_REQUESTS + 1000)
    u = torch.rand(n, generator=g).numpy()
    nk = torch.randint(0, 9, (n,), generator=g).numpy()
    sp = torch.randint(0, 2, (n,), generator=g).numpy()
    reqs = []
    for i in range(n):
        tenant = i % 2
        lo, hi = (0.0, 6.0) if tenant == 0 else (6.0, 12.0)       # log2 M
        M = max(1, int(round(2.0 ** (lo + (hi - lo) * u[i]))))
        reqs.append((tenant, M, SIZES[nk[i] // 3], SIZES[nk[i] % 3], bool(sp[i])))
    return reqs


def test_served_mix_sampled(gb, orc):
    from paper_2602_10262_gb300.server import Server
    dev = torch.device("cuda")
    reqs = _trace(48)
    used = sorted({(N, K) for _, _, N, K, _ in reqs})
    w_host, weights = {}, {}
    for j, (N, K) in enumerate(used):
        w = workloads.randn_f32((N, K), seed=500 + j)
        w_host[(N, K)] = w
        Wd, dW = gb.fp8_quantize_e4m3(torch.from_numpy(w).to(dev), 1)
        vals, meta = gb.prune24_compress(Wd)
        weights[(N, K)] = (Wd, dW, vals, meta)
    xs, outs, tickets = [], [], []
    with Server(num_tenants=2, latency_tenant=0, batching=True, pool_bytes=4 << 30) as srv:
        handles = {}
        for (N, K), (Wd, dW, vals, meta) in weights.items():
            handles[(N, K, False)] = srv.register_weight(N, K, Wd, dW, 1)
            handles[(N, K, True)] = srv.register_weight(N, K, vals, dW, 1, W_meta=meta)
        torch.cuda.synchronize()
        for i, (tenant, M, N, K, sp) in enumerate(reqs):
            xh = workloads.randn_f32((M, K), seed=1000 + i)
            x = torch.from_numpy(xh).to(dev)
            out = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device=dev)
            xs.append((xh, x))
            outs.append(out)
            tickets.append(srv.submit(tenant, handles[(N, K, sp)], M, x, K, out, N))
        res = [srv.wait(t, 120) for t in tickets]
        stats = srv.stats()
    assert all(r is not None and r.status == 0 for r in res)
    assert stats["completed"] == len(reqs)
    assert gb.fp8_last_device_error() == 0
    for i, (tenant, M, N, K, sp) in enumerate(reqs):
        ms, ns = sampled.entries(M, N, n=256, seed=700 + i, lines=False)
        x = xs[i][0]
        ref, S = sampled.reference(orc, x, w_host[(N, K)], ms, ns, sparse_w=sp)
        got = outs[i][torch.from_numpy(ms).to(dev), torch.from_numpy(ns).to(dev)].float().cpu().numpy()
        parity.check_bf16(got, ref, S, K)
