"""Benchmark of the FP8 E4M3 GEMM path on one or more GB300 GPUs.

One step = one pass of the hot path over one batch of synthetic input at
M = N = K (default 16384, the largest square shape of the dense sweep):
  quantise A [M,K] and B [N,K] from fp32 to E4M3 with per-row scales,
  2:4-prune A, dense FP8 GEMM (BF16 out), 2:4-sparse FP8 GEMM on the pruned
  A (BF16 out).
`value` = GEMM FLOPs of the step (2MNK dense + 2MNK sparse, dense-equivalent)
divided by the step time, summed over ranks (weak scaling: every rank runs
the same step on its own GPU; there is no data-path collective).

Prints one JSON line.  `--impl reference` times the CPU oracle instead (the
paper publishes no code; the oracle is the reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "FP8 GEMM TFLOP/s (% of peak), dense & 2:4; p99 latency batched vs per-call"
UNIT = "TFLOP/s"
FP8_PER_BF16 = 2.0          # nominal dense fp8 / bf16 tensor ratio (4.5 / 2.25 PFLOP/s)
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return FALLBACK, "fallback"


# ------------------------------------------------------------------ distributed

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ traffic record

def recorded_traffic(kernel_src: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (sha256 of the file recorded with it)."""
    path = os.path.join(ROOT, "profiles", f"gemm_fp8_kernel_{workload}.md")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.startswith("- "):
                k, v = line[2:].split(":", 1)
                rec[k.strip()] = v.strip().strip("`")
    src = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha256_16") != src:
        return None
    try:
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ oracle (CPU)

class OracleSample:
    """A sub-block of the step for the CPU oracle: rows [0, a) of A against
    rows [0, b) of B at full K, dense and 2:4-sparse.  Per-row scaling is
    row-local, so quantising only these rows gives the same codes as
    quantising the whole operands.  Inputs are produced by the oracle
    itself, outside the timed part."""

    def __init__(self, size: int, a: int, b: int, threads: int):
        import oracle
        self.orc = oracle.get()
        self.orc.set_threads(threads)
        self.size, self.a, self.b = size, a, b
        x = workloads.randn_f32((size, size), workloads.SEED_A)[:a]
        w = workloads.randn_f32((size, size), workloads.SEED_B)[:b]
        self.A, self.dA = self.orc.quantize(x, 1)
        self.B, self.dB = self.orc.quantize(w, 1)
        self.vals, self.meta = self.orc.prune24(self.A)

    def run(self):
        """Returns (FLOPs, seconds) of one dense + one sparse sub-block."""
        t0 = time.perf_counter()
        self.orc.gemm(self.A, self.B, self.dA, 1, self.dB, 1)
        self.orc.gemm_sparse24(self.vals, self.meta, self.B, self.size, self.dA, 1, self.dB, 1)
        dt = time.perf_counter() - t0
        return 2.0 * 2.0 * self.a * self.b * self.size, dt

    def describe(self):
        return (f"A rows [0,{self.a}) x B rows [0,{self.b}) at K={self.size}: "
                f"dense + 2:4 GEMM in FP64")


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    cores = cpu_cores()
    smp = OracleSample(args.size, 16, 256, cores)
    for _ in range(args.warmup):
        smp.run()
    total_f, total_t = 0.0, 0.0
    for _ in range(args.steps):
        f, t = smp.run()
        total_f += f
        total_t += t
    value = total_f / total_t / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1), torch.Generator)",
        "config": config(args.size, ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: " + smp.describe()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config(size, ws):
    return {"workload": f"fp8_e4m3_gemm_pipeline_{size}", "M": size, "N": size, "K": size,
            "scales": "per-row A, per-row B (per output channel)", "out": "bf16",
            "stages": "quantize A,B -> prune24 A -> dense GEMM -> 2:4 sparse GEMM",
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{ws}"}


# ------------------------------------------------------------------ GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=16384)
    ap.add_argument("--cpu-rows", type=int, default=512)
    ap.add_argument("--cpu-cols", type=int, default=2048)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import paper_2602_10262_gb300 as gb
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    gb.library()
    S = args.size
    M = N = K = S

    x_h = torch.from_numpy(workloads.randn_f32((M, K), workloads.SEED_A))
    w_h = torch.from_numpy(workloads.randn_f32((N, K), workloads.SEED_B))
    x = x_h.to(dev)
    w = w_h.to(dev)
    A = torch.empty((M, K), dtype=torch.uint8, device=dev)
    B = torch.empty((N, K), dtype=torch.uint8, device=dev)
    dA = torch.empty((M,), dtype=torch.float32, device=dev)
    dB = torch.empty((N,), dtype=torch.float32, device=dev)
    vals = torch.empty((M, K // 2), dtype=torch.uint8, device=dev)
    meta = torch.empty((M, K // 8), dtype=torch.uint8, device=dev)
    Cd = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
    Cs = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
    stream = torch.cuda.current_stream()

    # does this build have the sparse path?
    sparse_ok = True
    try:
        gb.fp8_quantize_e4m3(x, 1, A, dA)
        gb.prune24_compress(A, vals, meta)
        gb.fp8_quantize_e4m3(w, 1, B, dB)
        gb.gemm_fp8_sparse24(vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=Cs)
    except gb.Fp8Error as e:
        if e.status != -8:
            raise
        sparse_ok = False
    launches_per_step = 4 + (1 if sparse_ok else 0)

    ev = {}

    def step(record=None):
        if record is not None:
            record[0].record(stream)
        gb.fp8_quantize_e4m3(x, 1, A, dA)
        gb.fp8_quantize_e4m3(w, 1, B, dB)
        gb.prune24_compress(A, vals, meta)
        if record is not None:
            record[1].record(stream)
        gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=Cd)
        if record is not None:
            record[2].record(stream)
        if sparse_ok:
            gb.gemm_fp8_sparse24(vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=Cs)
        if record is not None:
            record[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if gb.fp8_last_device_error() != 0:
        raise RuntimeError("device error during warm-up")

    recs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        start.record(stream)
        for i in range(args.steps):
            step(recs[i])
        stop.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    ms_local = start.elapsed_time(stop)
    ms = max_over_ranks(ms_local, ws)
    if gb.fp8_last_device_error() != 0:
        raise RuntimeError("device error during the timed region")

    flops_dense = 2.0 * M * N * K
    flops_step = flops_dense * (2 if sparse_ok else 1)
    value = flops_step * args.steps * ws / (ms * 1e-3) / 1e12
    t_prep = np.mean([r[0].elapsed_time(r[1]) for r in recs])
    t_dense = np.mean([r[1].elapsed_time(r[2]) for r in recs])
    t_sparse = np.mean([r[2].elapsed_time(r[3]) for r in recs]) if sparse_ok else None

    pk, pk_kind = peaks()
    fp8_peak = pk["bf16_tflops"] * FP8_PER_BF16
    fp8_peak_sus = pk["bf16_tflops_sustained"] * FP8_PER_BF16
    dense_tflops = flops_dense / (t_dense * 1e-3) / 1e12
    roofline = {
        "bound": "tensor", "kernel": "gemm_fp8_kernel (dense)",
        "achieved": dense_tflops, "peak": fp8_peak, "unit": "TFLOP/s",
        "frac": dense_tflops / fp8_peak,
        "traffic": recorded_traffic(os.path.join(ROOT, "paper_2602_10262_gb300", "csrc", "gemm.cu"),
                                    f"dense_{S}"),
        "peak_note": f"{pk_kind}: bf16 burst {pk['bf16_tflops']} x {FP8_PER_BF16} (nominal fp8/bf16 ratio)",
        "frac_of_sustained": dense_tflops / fp8_peak_sus,
        "algorithmic_flops_per_launch": flops_dense,
    }
    stages = {"quantize_prune_ms": t_prep, "dense_ms": t_dense,
              "dense_tflops": dense_tflops}
    if sparse_ok:
        stages["sparse_ms"] = t_sparse
        stages["sparse_tflops_dense_equiv"] = flops_dense / (t_sparse * 1e-3) / 1e12
        stages["sparse_vs_dense_speedup"] = t_dense / t_sparse
    # quantise + prune traffic: read 2 x 4 B + write 2 x 1 B per element of A and
    # B (+ scales), prune reads 1 B and writes 0.625 B per element of A
    prep_bytes = (2 * 5.0 + 1.625) * M * K
    stages["quantize_prune_gbs"] = prep_bytes / (t_prep * 1e-3) / 1e9

    # ---------------------------------------------------------------- e2e
    e2e = None
    if not args.no_e2e:
        xp = x_h.pin_memory()
        wp = w_h.pin_memory()
        Cd_h = torch.empty((M, N), dtype=torch.bfloat16).pin_memory()
        Cs_h = torch.empty((M, N), dtype=torch.bfloat16).pin_memory()
        n_e2e = max(3, min(args.steps, 10))

        def e2e_step():
            x.copy_(xp, non_blocking=True)
            w.copy_(wp, non_blocking=True)
            step()
            Cd_h.copy_(Cd, non_blocking=True)
            if sparse_ok:
                Cs_h.copy_(Cs, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(n_e2e):
            e2e_step()
        s1.record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        ms_e2e = max_over_ranks(s0.elapsed_time(s1), ws)
        h2d = (x_h.numel() + w_h.numel()) * 4
        d2h = M * N * 2 * (2 if sparse_ok else 1)
        e2e = {"value": flops_step * n_e2e * ws / (ms_e2e * 1e-3) / 1e12, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": ms_e2e / n_e2e, "steps": n_e2e,
               "path": "pinned host fp32 -> H2D -> C ABI (quantize, prune, dense, sparse) -> D2H bf16"}

    # ---------------------------------------------------------------- CPU oracle
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cores = cpu_cores()
        smp = OracleSample(S, args.cpu_rows, args.cpu_cols, cores)
        f, t = smp.run()
        cpu = {"value": f / t / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": smp.describe() + f", {t:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "e4m3 (fp32 accumulate)",
            "data": "synthetic (seeded N(0,1) fp32, torch.Generator)",
            "config": config(S, ws),
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "stages": stages, "sparse_path": sparse_ok,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks.summary(),
        }
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
