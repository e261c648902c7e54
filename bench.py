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
    """SM clock and clock-event (throttle) reasons sampled during a region:
    every 5 ms through NVML (the driver's libnvidia-ml.so.1, read only),
    else every 100 ms from nvidia-smi."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # nvmlClocksEventReason bits (nvml.h)
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                   "hw_thermal_slowdown": 0x40, "hw_power_brake_slowdown": 0x80}
    PERIOD_S = 0.005

    def __init__(self, index: int, uuid: str = None):
        self.index = index
        self.uuid = uuid           # CUDA and NVML may number GPUs differently
        self.proc = None
        self.lines = []
        self.samples = []          # (sm_mhz, reason bits) from NVML
        self.max_mhz = None
        self.nvml = None
        self.stop = threading.Event()

    def _nvml_open(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            if self.uuid:
                rc = lib.nvmlDeviceGetHandleByUUID(ctypes.c_char_p(self.uuid.encode()), ctypes.byref(h))
            else:
                rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h))
            if rc != 0:
                return None
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:      # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            return lib, h
        except OSError:
            return None

    def _nvml_loop(self):
        import ctypes
        lib, h = self.nvml
        clk, why = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and \
                    lib.nvmlDeviceGetCurrentClocksEventReasons(h, ctypes.byref(why)) == 0:
                self.samples.append((float(clk.value), int(why.value)))
            self.stop.wait(self.PERIOD_S)

    def __enter__(self):
        self.nvml = self._nvml_open()
        if self.nvml is not None:
            self.thread = threading.Thread(target=self._nvml_loop, daemon=True)
            self.thread.start()
            return self
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
        if self.nvml is not None:
            self.stop.set()
            self.thread.join(timeout=5)
            try:
                self.nvml[0].nvmlShutdown()
            except Exception:
                pass
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if self.nvml is not None:
            sm = [c for c, _ in self.samples]
            reasons = sorted(n for n, bit in self.REASON_BITS.items() if any(w & bit for _, w in self.samples))
            return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": self.max_mhz,
                    "reasons": reasons, "samples": len(sm), "source": "nvml, 5 ms"}
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
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 100 ms"}


def gpu_uuid(dev):
    """NVML's UUID string of a CUDA device ("GPU-..."), or None."""
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None
    return u if u.startswith("GPU-") else "GPU-" + u


# ------------------------------------------------------------------ traffic record

def recorded_traffic(kernel_src: str, workload: str, profiles_dir: str = None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (sha256 of the file recorded with it)."""
    path = os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), f"gemm_fp8_kernel_{workload}.md")
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

    def run(self, a=None, b=None):
        """Returns (FLOPs, seconds) of one dense + one sparse sub-block (the
        first a rows of A and b rows of B; default: all of the sample).  The
        full sub-block's results are kept for check()."""
        a = self.a if a is None else min(a, self.a)
        b = self.b if b is None else min(b, self.b)
        t0 = time.perf_counter()
        Cd = self.orc.gemm(self.A[:a], self.B[:b], self.dA[:a], 1, self.dB[:b], 1)
        Cs = self.orc.gemm_sparse24(self.vals[:a], self.meta[:a], self.B[:b], self.size, self.dA[:a], 1,
                                    self.dB[:b], 1)
        dt = time.perf_counter() - t0
        if a == self.a and b == self.b:
            self.ref = (Cd, Cs)
        return 2.0 * 2.0 * a * b * self.size, dt

    def _bf16_check(self, got, ref, A):
        """The BF16 bound per element, |C - ref| <= 1e-2 |ref| + gamma S with
        S = dA dB sum_k |a b| and gamma = (K + 2) 2^-24 (S from the oracle's
        decoded codes)."""
        dec = lambda c: self.orc.decode(c & np.uint8(0x7F), 0)
        S = (dec(A) @ dec(self.B).T) * np.abs(self.dA.astype(np.float64))[:, None] \
            * np.abs(self.dB.astype(np.float64))[None, :]
        gamma = (self.size + 2) * 2.0 ** -24
        diff = np.abs(got.astype(np.float64) - ref)
        bound = 1e-2 * np.abs(ref) + gamma * S
        return {"elements": int(ref.size), "failed": int(np.count_nonzero(diff > bound)),
                "needed_gamma_term": int(np.count_nonzero(diff > 1e-2 * np.abs(ref))),
                "max_err_over_bound": float(np.max(diff / bound)),
                "normwise_rel_err": float(np.linalg.norm(got.astype(np.float64) - ref) / np.linalg.norm(ref))}

    def check(self, gpu):
        """The GPU step's codes, scales, compressed A and outputs on this
        sub-block against the oracle's (gpu: host copies of the same rows)."""
        Cd, Cs = self.ref
        out = {"sub_block": f"rows [0,{self.a}) of A x rows [0,{self.b}) of B, K={self.size}",
               "quantize_bitexact": bool(np.array_equal(gpu["A"], self.A) and np.array_equal(gpu["B"], self.B)
                                         and np.array_equal(gpu["dA"], self.dA)
                                         and np.array_equal(gpu["dB"], self.dB)),
               "prune_bitexact": bool(np.array_equal(gpu["vals"], self.vals)
                                      and np.array_equal(gpu["meta"], self.meta)),
               "dense": self._bf16_check(gpu["Cd"], Cd, self.A),
               "sparse": self._bf16_check(gpu["Cs"], Cs, self.orc.decompress24(self.vals, self.meta, self.size)),
               "tolerance": "bf16: |C - ref| <= 1e-2 |ref| + (K+2) 2^-24 dA dB sum|a b| per element"}
        out["pass"] = (out["quantize_bitexact"] and out["prune_bitexact"] and out["dense"]["failed"] == 0
                       and out["sparse"]["failed"] == 0)
        return out

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
            "stages": "quantize + 2:4-compress A (one pass), quantize B -> dense GEMM -> 2:4 sparse GEMM",
            "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{ws}"}


# ------------------------------------------------------------------ serving

class ServingBench:
    """Poisson stream of FP8 GEMM requests from two tenants against resident
    weights, served by the library's request server.  Modes: per call (one
    quantise + one GEMM launch per request: the baseline), continuous
    batching with the latency tenant's requests launched as they arrive and
    the bulk tenant's GEMMs leaving `reserve` SMs free for them (the
    server's policy, "batched"), and continuous batching without a reserve.

    Tenant 0 (latency): M log-uniform in [1, 64]; tenant 1 (throughput): M
    log-uniform in [64, 4096]; (N, K) uniform over {4096, 8192, 14336}^2;
    half the requests use the 2:4-sparse copy of the weight.  Inputs are
    seeded synthetic fp32 (seed 2 for the trace); each request reads its
    activations from a random row offset of a 16384-row buffer.  Every
    request in flight has an output slot of its own (no two in-flight
    requests write the same bytes); a slot is reused once its request's
    result has been collected."""

    SIZES = (4096, 8192, 14336)
    RESERVE = 16                   # SMs the batched mode keeps free for the latency tenant
    SLOTS = 128                    # output slots (requests in flight at most)

    def __init__(self, dev, gb):
        self.gb, self.dev = gb, dev
        g = torch.Generator(device=dev).manual_seed(workloads.SEED_REQUESTS)
        self.weights = {}
        for N in self.SIZES:
            for K in self.SIZES:
                w = torch.randn((N, K), generator=g, device=dev, dtype=torch.float32)
                Wd, dW = gb.fp8_quantize_e4m3(w, 1)
                vals, meta = gb.prune24_compress(Wd)
                self.weights[(N, K)] = (Wd, dW, vals, meta)
                del w
        self.X = torch.randn((16384, max(self.SIZES)), generator=g, device=dev, dtype=torch.float32)
        self.slot_elems = 4096 * max(self.SIZES)
        self.outs = torch.empty((self.SLOTS, self.slot_elems), dtype=torch.bfloat16, device=dev)
        torch.cuda.synchronize()

    def trace(self, n, seed):
        rng = np.random.default_rng(seed)
        tenant = rng.integers(0, 2, n)
        u = rng.random(n)
        M = np.where(tenant == 0, np.round(2.0 ** (u * 6.0)), np.round(2.0 ** (6.0 + u * 6.0)))
        N = rng.choice(self.SIZES, n)
        K = rng.choice(self.SIZES, n)
        sparse = rng.random(n) < 0.5
        gap = rng.exponential(1.0, n)           # unit-rate Poisson arrivals, scaled later
        row = rng.integers(0, 16384 - 4096, n)  # activation rows [row, row + M)
        return [dict(tenant=int(t), M=int(m), N=int(nn), K=int(k), sparse=bool(sp), gap=float(gp), row=int(r0))
                for t, m, nn, k, sp, gp, r0 in zip(tenant, M, N, K, sparse, gap, row)]

    LATENCY_POOL = 1 << 30         # pool bytes the bulk tenant leaves to the latency tenant

    def modes(self):
        sms = self.gb.fp8_device_sm_count()
        return {"per_call": dict(batching=False),
                "batched": dict(batching=True, bulk_max_ctas=max(sms - self.RESERVE, 1),
                                latency_pool_bytes=self.LATENCY_POOL),
                "batched_no_reserve": dict(batching=True, latency_pool_bytes=self.LATENCY_POOL)}

    def _server(self, mode_cfg):
        from paper_2602_10262_gb300.server import Server
        cfg = dict(mode_cfg)
        pool = cfg.pop("pool_bytes", 8 << 30)
        srv = Server(num_tenants=2, latency_tenant=0, pool_bytes=pool, **cfg)
        handles = {}
        for (N, K), (Wd, dW, vals, meta) in self.weights.items():
            handles[(N, K, False)] = srv.register_weight(N, K, Wd, dW, 1)
            handles[(N, K, True)] = srv.register_weight(N, K, vals, dW, 1, W_meta=meta)
        return srv, handles

    def run(self, reqs, mode_cfg, rate=None, window=96):
        """Serve `reqs`: Poisson arrivals at `rate` requests/s, or (rate None)
        a closed loop keeping `window` requests in flight.  Returns latencies
        (us), the makespan (us), the server's stats and the results."""
        from collections import deque
        srv, handles = self._server(mode_cfg)
        ld = self.X.stride(0)
        xb, ob = self.X.data_ptr(), self.outs.data_ptr()
        free = list(range(self.SLOTS))
        pend = (deque(), deque())                # per tenant: (ticket, slot, index), in order
        res = [None] * len(reqs)
        inflight = 0

        def collect(block):
            nonlocal inflight
            got = False
            for q in pend:
                while q:
                    t, slot, i = q[0]
                    r = srv.wait(t, 60) if block and not got else srv.poll(t)
                    if r is None:
                        break
                    q.popleft()
                    res[i] = r
                    free.append(slot)
                    inflight -= 1
                    got = True
            return got

        import gc
        lag = np.zeros(len(reqs))
        gc_was = gc.isenabled()
        gc.disable()                 # a collector pause would bunch the Poisson arrivals
        try:
            times = None
            if rate is not None:
                times = np.cumsum([r["gap"] for r in reqs]) / rate * 1e6
            t0 = srv.now_us() + 1000.0
            for i, r in enumerate(reqs):
                if times is not None:
                    target = t0 + times[i]
                    while srv.now_us() < target:
                        collect(False)
                    lag[i] = srv.now_us() - target
                while not free or (rate is None and inflight >= window):
                    if not collect(False):
                        oldest = min((q for q in pend if q), key=lambda q: q[0][2])
                        r0 = srv.wait(oldest[0][0], 60)
                        t_, slot, j = oldest.popleft()
                        res[j] = r0
                        free.append(slot)
                        inflight -= 1
                slot = free.pop()
                x = xb + 4 * r["row"] * ld
                tk = srv.submit(r["tenant"], handles[(r["N"], r["K"], r["sparse"])], r["M"], x, ld,
                                ob + 2 * slot * self.slot_elems, r["N"])
                pend[r["tenant"]].append((tk, slot, i))
                inflight += 1
            while inflight:
                collect(True)
            stats = srv.stats()
        finally:
            srv.close()
            if gc_was:
                gc.enable()
        # how late the generator submitted (open loop: late submissions bunch up)
        stats["submit_lag_us"] = {"p50": float(np.percentile(lag, 50)), "p99": float(np.percentile(lag, 99)),
                                  "max": float(lag.max())}
        if any(x is None or x.status != 0 for x in res):
            raise RuntimeError("serving request failed")
        lat = np.array([x.t_end_us - x.t_submit_us for x in res])
        first = min(x.t_submit_us for x in res)
        last = max(x.t_end_us for x in res)
        return lat, last - first, stats, res

    @staticmethod
    def flops(reqs):
        return sum(2.0 * r["M"] * r["N"] * r["K"] for r in reqs)

    def isolated(self, reqs):
        """Latency of each request run alone (per-call server, one at a time)."""
        srv, handles = self._server(dict(batching=False))
        ld = self.X.stride(0)
        out = []
        try:
            for r in reqs:
                t = srv.submit(r["tenant"], handles[(r["N"], r["K"], r["sparse"])], r["M"],
                               self.X.data_ptr() + 4 * r["row"] * ld, ld, self.outs.data_ptr(), r["N"])
                x = srv.wait(t, 60)
                out.append(x.t_end_us - x.t_submit_us)
        finally:
            srv.close()
        return np.array(out)


def serving_report(gb, dev, n_cap=20000, n_load=20000, loads=(0.8,), n_iso=2000):
    """Capacity of each serving mode (closed loop, 96 requests in flight),
    then the same seeded Poisson trace of n_load requests offered at each
    fraction of the lowest capacity in `loads`.  Slowdown = latency / the
    request's latency alone, measured for the first n_iso requests; Jain's
    index and the paper's fairness 1 - (max - min) / mean and min / max are
    taken over the tenants' mean slowdowns (tenants of very different sizes
    are compared by how much the mix slows each down).  The first load's
    results sit at the top level; further loads under "other_loads"."""
    from paper_2602_10262_gb300.server import overlap_efficiency
    sb = ServingBench(dev, gb)
    modes = sb.modes()
    cap_reqs = sb.trace(n_cap, workloads.SEED_REQUESTS + 1)
    cap = {}
    for mode, cfg in modes.items():
        sb.run(cap_reqs[:256], cfg)                          # warm-up
        _, span, stats, _ = sb.run(cap_reqs, cfg)
        cap[mode] = {"tflops": sb.flops(cap_reqs) / (span * 1e-6) / 1e12,
                     "req_per_s": n_cap / (span * 1e-6),
                     "kernel_launches": stats["kernel_launches"], "batches": stats["batches"]}
    reqs = sb.trace(n_load, workloads.SEED_REQUESTS)
    iso = sb.isolated(reqs[:n_iso])
    tenant = np.array([r["tenant"] for r in reqs])
    out = {"workload": "Poisson two-tenant GEMM stream, M log-uniform [1,4096], "
                       "(N,K) in {4096,8192,14336}^2, 50% 2:4-sparse weights",
           "requests_per_point": n_load, "modes": {m: {k: v for k, v in c.items()} for m, c in modes.items()},
           "capacity": cap}
    for i, load in enumerate(loads):
        base = min(cap, key=lambda m: cap[m]["req_per_s"])
        rate = load * cap[base]["req_per_s"]
        block = {"offered_load": f"{load} x {base} capacity = {rate:.0f} req/s"}
        for mode, cfg in modes.items():
            lat, span, stats, res = sb.run(reqs, cfg, rate)
            slow = lat[:n_iso] / iso
            t_iso = tenant[:n_iso]
            x = [float(np.mean(slow[t_iso == t])) for t in (0, 1)]              # mean slowdown
            y = [float(np.mean(1.0 / slow[t_iso == t])) for t in (0, 1)]        # isolated / observed
            block[mode] = {
                "p50_us": {f"tenant{t}": float(np.percentile(lat[tenant == t], 50)) for t in (0, 1)},
                "p99_us": {f"tenant{t}": float(np.percentile(lat[tenant == t], 99)) for t in (0, 1)},
                "p99_all_us": float(np.percentile(lat, 99)),
                "mean_slowdown": {f"tenant{t}": x[t] for t in (0, 1)},
                "tflops": sb.flops(reqs) / (span * 1e-6) / 1e12,
                "jain": (sum(y) ** 2) / (2 * sum(v * v for v in y)),
                "fairness_1_minus_range_over_mean": 1.0 - (max(x) - min(x)) / np.mean(x),
                "fairness_min_over_max": min(x) / max(x),
                "overlap_efficiency": overlap_efficiency(res),
                "mean_batch": float(np.mean([r.batch_size for r in res])),
                "max_batch": int(stats["max_batch_seen"]),
                "pool_high_water_mb": stats["pool_high_water"] / 2 ** 20,
                "submit_lag_us": stats["submit_lag_us"],
                "kernel_launches": stats["kernel_launches"],
            }
        if i == 0:
            out.update(block)
        else:
            out.setdefault("other_loads", {})[str(load)] = block
    return out


def _l2_copies(dev, set_bytes):
    """Operand sets to rotate through so that one pass streams at least twice
    the L2 capacity: every timed call then starts with its operands outside
    L2 (as a weight read once per step would)."""
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    return max(1, min(64, -(-2 * l2 // max(1, set_bytes))))


def _time_ms(fn, target_s=0.15, warmup=3, reps=10, capture=True):
    """Device time per call of fn (a callable, or a list of callables taken
    in turn, each counting as one call): `reps` rounds are captured in a
    CUDA graph (the library's launches and cuBLAS both capture) and the
    graph is replayed, so host-side call overhead does not hide in the
    number.  capture=False times fn itself (for fn that already replays a
    graph)."""
    fns = fn if isinstance(fn, (list, tuple)) else [fn]
    for _ in range(warmup):
        for f in fns:
            f()
    torch.cuda.synchronize()
    if not capture:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            for f in fns:
                f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / (20 * len(fns))
    reps = max(1, reps // len(fns))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=s):
        for _ in range(reps):
            for f in fns:
                f()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.replay()
    e1.record()
    torch.cuda.synchronize()
    one = max(e0.elapsed_time(e1), 1e-3)
    n = max(3, min(200, int(target_s * 1e3 / one)))
    e0.record()
    for _ in range(n):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (n * reps * len(fns))
    del g
    return ms


def _operands(gb, M, N, K, dev, seed, a_fmt=0, b_fmt=0):
    g = torch.Generator(device=dev).manual_seed(seed)
    x = torch.randn((M, K), generator=g, device=dev)
    w = torch.randn((N, K), generator=g, device=dev)
    quant = {0: gb.fp8_quantize_e4m3, 1: gb.fp8_quantize_e5m2}
    A, dA = quant[a_fmt](x, 1)
    B, dB = quant[b_fmt](w, 1)
    return x, w, A, dA, B, dB


FORMAT_NAMES = {0: "e4m3", 1: "e5m2"}


def occupancy_sweep(gb, dev, peak_fp8):
    """Throughput against the number of CTAs of the persistent kernel (one
    CTA per SM), for one fixed dense and one fixed 2:4 GEMM: the analogue of
    the paper's throughput-vs-active-wavefronts sweep (section 4.2), with
    the grid capped through gemm_fp8_grouped_ex."""
    M = N = K = 8192
    sms = gb.fp8_device_sm_count()
    caps = sorted({c for c in (1, 2, 4, 8, 16, 32, 64, 76, 96, 128, sms) if c <= sms})
    x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 4242)
    del x, w
    vals, meta = gb.prune24_compress(A)
    n8 = _l2_copies(dev, M * K + N * K + 2 * M * N)
    sets = []
    for i in range(n8):
        a, b, v, m = (A, B, vals, meta) if i == 0 else (A.clone(), B.clone(), vals.clone(), meta.clone())
        C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
        sets.append((a, b, v, m, C, [gb.make_problem(a, b, dA, 1, dB, 1, C, 1.0, gb.OUT_BF16)],
                     [gb.make_problem(v, b, dA, 1, dB, 1, C, 1.0, gb.OUT_BF16, A_meta=m)]))
    rows = []
    flops = 2.0 * M * N * K
    for cap in caps:
        row = {"ctas": cap}
        for kind, idx in (("dense", 5), ("sparse", 6)):
            ms = _time_ms([lambda p=st[idx]: gb.gemm_fp8_grouped_ex(p, cap) for st in sets])
            row[f"{kind}_ms"] = ms
            row[f"{kind}_tflops"] = flops / ms / 1e9
            row[f"{kind}_frac_of_peak"] = flops / ms / 1e9 / peak_fp8
        rows.append(row)
    del sets
    torch.cuda.empty_cache()
    return {"M": M, "N": N, "K": K, "peak_fp8_tflops": peak_fp8, "operand_copies": n8,
            "rows": rows}


class _Span:
    def __init__(self, a, b):
        self.t_start_us, self.t_end_us = a, b


def _concurrent(graphs, streams):
    """Replay graphs[i] on streams[i], all released together by one event;
    returns (per-stream [start, end] in ms from the release, makespan ms)."""
    cur = torch.cuda.current_stream()
    go = torch.cuda.Event(enable_timing=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in graphs]
    ends = [torch.cuda.Event(enable_timing=True) for _ in graphs]
    torch.cuda.synchronize()
    go.record(cur)
    for g, st, e0, e1 in zip(graphs, streams, starts, ends):
        st.wait_event(go)
        with torch.cuda.stream(st):
            e0.record(st)
            g.replay()
            e1.record(st)
    for st in streams:
        cur.wait_stream(st)
    torch.cuda.synchronize()
    spans = [(go.elapsed_time(a), go.elapsed_time(b)) for a, b in zip(starts, ends)]
    return spans, max(b for _, b in spans)


def _capture(fn, iters, stream):
    """fn(stream) `iters` times captured into one CUDA graph on `stream`."""
    with torch.cuda.stream(stream):
        for _ in range(3):
            fn(stream)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(iters):
            fn(stream)
    torch.cuda.synchronize()
    return g


def _concurrency_stats(spans, makespan, iso_ms):
    """The paper's concurrency metrics (sections 3.2, 5, 6.2) for one run:
    speedup = serial time of the same work / makespan; per-stream times,
    their CV, fairness 1 - (max - min) / mean and min / max; overlap
    efficiency = share of busy time with two or more streams active."""
    from paper_2602_10262_gb300.server import overlap_efficiency
    t = np.array([b - a for a, b in spans])
    return {"streams": len(spans), "makespan_ms": makespan, "serial_ms": float(sum(iso_ms)),
            "speedup": float(sum(iso_ms) / makespan),
            "per_stream_ms": [float(v) for v in t],
            "per_stream_speedup": [float(i / v) for i, v in zip(iso_ms, t)],
            "cv": float(t.std() / t.mean()), "fairness_1_minus_range_over_mean":
                float(1.0 - (t.max() - t.min()) / t.mean()),
            "fairness_min_over_max": float(t.min() / t.max()),
            "overlap_efficiency": overlap_efficiency([_Span(a * 1e3, b * 1e3) for a, b in spans],
                                                     one_per_interval=False)}


def concurrency_sweep(gb, dev, iters=100, trials=5):
    """The paper's concurrency experiments replayed on GB300 streams: each
    stream replays a CUDA graph of `iters` GEMMs (so host issue does not
    limit it), all streams released by one event; medians over `trials`.
      - streams: 1, 2, 4, 8 streams of 512^3 GEMMs, FP8 dense, FP8 2:4 and
        BF16 torch.matmul (section 5.1), and dense/sparse alternating
        ("mixed", section 6.2);
      - fragmentation: pairs 512^3 + 512^3, 1024^3 + 512^3, 2048^3 + 512^3
        (section 5.3), sharing the SMs freely and with 24 SMs reserved for
        the small stream (the larger GEMM's grid capped at SMs - 24 through
        gemm_fp8_grouped_ex, as the server's co-scheduled mode does;
        occupancy-aware co-scheduling, section 8.2);
      - transformer: two instances of the transformer layer (grouped,
        graph-captured) on two streams against one after the other
        (section 7.2)."""
    sms = gb.fp8_device_sm_count()
    streams = [torch.cuda.Stream() for _ in range(8)]
    keep = []

    def dense_fn(n, seed, max_ctas=0):
        x, w, A, dA, B, dB = _operands(gb, n, n, n, dev, seed)
        C = torch.empty((n, n), dtype=torch.bfloat16, device=dev)
        keep.extend([A, dA, B, dB, C])
        pr = [gb.make_problem(A, B, dA, 1, dB, 1, C, 1.0, gb.OUT_BF16)]
        return lambda st: gb.gemm_fp8_grouped_ex(pr, max_ctas, stream=st)

    def sparse_fn(n, seed):
        x, w, A, dA, B, dB = _operands(gb, n, n, n, dev, seed)
        vals, meta = gb.prune24_compress(A)
        C = torch.empty((n, n), dtype=torch.bfloat16, device=dev)
        keep.extend([vals, meta, dA, B, dB, C])
        return lambda st: gb.gemm_fp8_sparse24(vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=C,
                                               stream=st)

    def bf16_fn(n, seed):
        g = torch.Generator(device=dev).manual_seed(seed)
        xb = torch.randn((n, n), generator=g, device=dev).bfloat16()
        wb = torch.randn((n, n), generator=g, device=dev).bfloat16()
        C = torch.empty((n, n), dtype=torch.bfloat16, device=dev)
        keep.extend([xb, wb, C])
        return lambda st: torch.matmul(xb, wb.T, out=C)

    def run(fns, iso=None, n_iter=iters):
        graphs = [_capture(f, n_iter, streams[i]) for i, f in enumerate(fns)]
        if iso is None:                                  # each graph alone
            iso = [float(np.median([_concurrent([g], [streams[i]])[1] for _ in range(trials)]))
                   for i, g in enumerate(graphs)]
        _concurrent(graphs, streams[:len(graphs)])       # warm-up
        res = [_concurrency_stats(*_concurrent(graphs, streams[:len(graphs)]), iso)
               for _ in range(trials)]
        med = {}
        for k, v in res[0].items():
            if isinstance(v, float):
                med[k] = float(np.median([r[k] for r in res]))
            elif isinstance(v, list):
                med[k] = [float(np.median([r[k][i] for r in res])) for i in range(len(v))]
            else:
                med[k] = v
        del graphs
        return med, iso

    out = {"iters_per_stream": iters, "trials": trials, "streams": [], "fragmentation": []}
    n = 512
    makers = {"fp8_dense": lambda i: dense_fn(n, 1000 + i), "fp8_sparse": lambda i: sparse_fn(n, 1000 + i),
              "bf16": lambda i: bf16_fn(n, 1000 + i),
              "fp8_mixed": lambda i: dense_fn(n, 1000 + i) if i % 2 == 0 else sparse_fn(n, 1000 + i)}
    for kind, mk in makers.items():
        fns = [mk(i) for i in range(4 if kind == "fp8_mixed" else 8)]
        for ns in (1, 2, 4, 8):
            if ns > len(fns):
                continue
            med, _ = run(fns[:ns])
            med.update({"kind": kind, "n": n, "gflops_aggregate": 2.0 * n ** 3 * iters * ns / med["makespan_ms"] / 1e6})
            out["streams"].append(med)
    reserve = min(24, sms // 2)
    for big in (512, 1024, 2048):
        for mode, caps in (("shared", (0, 0)), ("reserved", (sms - reserve, reserve))):
            fns = [dense_fn(big, 2000 + big, caps[0]), dense_fn(n, 2001, caps[1])]
            iso = None
            if mode == "reserved":
                iso = out["fragmentation"][-1]["isolated_ms"]      # uncapped, alone
            med, iso = run(fns, iso)
            med.update({"pair": [big, n], "ratio": f"{big // n}:1",
                        "mode": mode, "ctas": list(caps), "isolated_ms": iso})
            out["fragmentation"].append(med)
    # two transformer-layer instances
    inst = []
    flops = 0.0
    for r in range(2):
        probs = []
        for i, (name, M, N, K) in enumerate(workloads.TRANSFORMER_LAYER):
            x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 3000 + 10 * r + i)
            del x, w
            C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
            keep.extend([A, dA, B, dB, C])
            probs.append(gb.make_problem(A, B, dA, 1, dB, 1, C, 1.0, gb.OUT_BF16))
            if r == 0:
                flops += 2.0 * M * N * K
        inst.append(lambda st, p=probs: gb.gemm_fp8_grouped(p, stream=st))
    tf_iters = 10
    med, iso = run(inst, n_iter=tf_iters)
    med.update({"gflop_per_layer": flops / 1e9, "layers_per_instance": tf_iters,
                "aggregate_tflops": 2 * flops * tf_iters / med["makespan_ms"] / 1e9,
                "isolated_ms": iso})
    out["transformer_two_instances"] = med
    del keep
    torch.cuda.empty_cache()
    return out


def served_concurrency_sweep(gb, dev, iters=100, trials=3):
    """The paper's concurrency experiments (sections 5.1, 5.3, 6.2, 7.2)
    replayed as tenants of the request server (fp8_server_*): each tenant
    submits its `iters` requests at once (fp32 activations quantised per row
    by the server, resident E4M3 weights, BF16 out) and the server runs them
    one launch per request on the tenant's stream, as the paper's streams
    issue one GEMM after another; medians over `trials`.
      - tenants: 1, 2, 4, 8 tenants of 512^3 requests, dense, 2:4 and
        alternating dense / 2:4 (sections 5.1, 6.2); the dense sweep also
        with continuous batching;
      - fragmentation (section 5.3): a 512^3 tenant beside a 512^3, 1024^3
        or 2048^3 tenant, sharing every SM, or with the 512^3 tenant as the
        server's latency tenant (high-priority stream) and the larger one's
        GEMMs capped at SMs - 24 CTAs (bulk_max_ctas);
      - two transformer-layer instances (section 7.2): two tenants each
        submitting the four layer GEMMs 10 times.
    A tenant's time runs from its first submission to its last completion;
    its isolated time is the same requests alone on the same server
    configuration; overlap efficiency is over the tenants' spans."""
    from paper_2602_10262_gb300.server import Server
    sms = gb.fp8_device_sm_count()
    g = torch.Generator(device=dev).manual_seed(4000)
    weights = {}

    def weight(N, K, sparse):
        key = (N, K, sparse)
        if key not in weights:
            w = torch.randn((N, K), generator=g, device=dev)
            Wd, dW = gb.fp8_quantize_e4m3(w, 1)
            if sparse:
                vals, meta = gb.prune24_compress(Wd)
                weights[key] = (vals, dW, meta)
            else:
                weights[key] = (Wd, dW, None)
            del w
        return weights[key]

    X = torch.randn((16384, 14336), generator=g, device=dev)
    ld = X.stride(0)

    def serve(tenants, cfg, reuse_outputs=False):
        """tenants: per tenant a list of (M, N, K, sparse); all requests are
        submitted at once, interleaved over the tenants.  Returns per-tenant
        (start, end) spans and the makespan, in ms."""
        srv = Server(num_tenants=len(tenants), pool_bytes=16 << 30, **cfg)
        outs, tickets = [], [[] for _ in tenants]
        try:
            handles = {}
            for reqs in tenants:
                for (M, N, K, sp) in reqs:
                    if (N, K, sp) not in handles:
                        W, dW, meta = weight(N, K, sp)
                        handles[(N, K, sp)] = srv.register_weight(N, K, W, dW, 1, W_meta=meta)
            bufs = {}
            for t, reqs in enumerate(tenants):
                for i, (M, N, K, sp) in enumerate(reqs):
                    key = (t, M, N) if reuse_outputs else (t, i)
                    if key not in bufs:
                        bufs[key] = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
            torch.cuda.synchronize()
            n = max(len(r) for r in tenants)
            for i in range(n):
                for t, reqs in enumerate(tenants):
                    if i < len(reqs):
                        M, N, K, sp = reqs[i]
                        out = bufs[(t, M, N) if reuse_outputs else (t, i)]
                        tickets[t].append(srv.submit(t, handles[(N, K, sp)], M, X.data_ptr(), ld,
                                                     out.data_ptr(), N))
            res = [[srv.wait(tk, 120) for tk in tks] for tks in tickets]
        finally:
            srv.close()
        if any(r is None or r.status != 0 for rs in res for r in rs):
            raise RuntimeError("served concurrency request failed")
        spans = [(min(r.t_submit_us for r in rs) * 1e-3, max(r.t_end_us for r in rs) * 1e-3) for rs in res]
        make = max(b for _, b in spans) - min(a for a, _ in spans)
        return spans, make

    def measure(tenants, cfg, iso_cfgs=None, reuse_outputs=False):
        serve(tenants, cfg, reuse_outputs)                           # warm-up
        iso = []
        for t, reqs in enumerate(tenants):
            c = (iso_cfgs or [cfg] * len(tenants))[t]
            one = [float(np.median([(lambda s: s[1])(serve([reqs], c, reuse_outputs))
                                    for _ in range(trials)]))]
            iso += one
        runs = [_concurrency_stats(*serve(tenants, cfg, reuse_outputs), iso) for _ in range(trials)]
        med = {}
        for k, v in runs[0].items():
            if isinstance(v, float):
                med[k] = float(np.median([r[k] for r in runs]))
            elif isinstance(v, list):
                med[k] = [float(np.median([r[k][i] for r in runs])) for i in range(len(v))]
            else:
                med[k] = v
        med["isolated_ms"] = iso
        return med

    out = {"iters_per_tenant": iters, "trials": trials, "tenants": [], "fragmentation": []}
    n = 512
    kinds = {"fp8_dense": lambda i: False, "fp8_sparse": lambda i: True, "fp8_mixed": lambda i: i % 2 == 1}
    for kind, sp_of in kinds.items():
        for nt in (1, 2, 4, 8):
            if kind == "fp8_mixed" and nt > 4:
                continue
            tenants = [[(n, n, n, sp_of(t))] * iters for t in range(nt)]
            for batching in ((False, True) if kind == "fp8_dense" else (False,)):
                med = measure(tenants, dict(latency_tenant=-1, batching=batching))
                med.update({"kind": kind, "n": n, "batching": batching,
                            "gflops_aggregate": 2.0 * n ** 3 * iters * nt / med["makespan_ms"] / 1e6})
                out["tenants"].append(med)
    reserve = min(24, sms // 2)
    for big in (512, 1024, 2048):
        tenants = [[(big, big, big, False)] * iters, [(n, n, n, False)] * iters]
        for mode, cfg in (("shared", dict(latency_tenant=-1)),
                          ("reserved", dict(latency_tenant=1, bulk_max_ctas=sms - reserve))):
            med = measure(tenants, cfg, iso_cfgs=[dict(latency_tenant=-1)] * 2)
            med.update({"pair": [big, n], "ratio": f"{big // n}:1", "mode": mode})
            out["fragmentation"].append(med)
    layer = [(M, N, K, False) for _, M, N, K in workloads.TRANSFORMER_LAYER]
    flops = sum(2.0 * M * N * K for M, N, K, _ in layer)
    tf_iters = 10
    med = measure([layer * tf_iters, layer * tf_iters], dict(latency_tenant=-1), reuse_outputs=True)
    med.update({"gflop_per_layer": flops / 1e9, "layers_per_instance": tf_iters,
                "aggregate_tflops": 2 * flops * tf_iters / med["makespan_ms"] / 1e9})
    out["transformer_two_instances"] = med
    del X, weights
    torch.cuda.empty_cache()
    return out


def aspect_sweep(gb, dev):
    """Throughput against the aspect ratio M/N at fixed work (M * N = 8192^2
    outputs, K = 4096): the analogue of the paper's shape sweep at fixed
    total blocks (section 4.3).  FP8 dense against BF16 torch.matmul."""
    K = 4096
    rows = []
    for lg in (-6, -4, -2, 0, 2, 4, 6):
        M = int(8192 * 2.0 ** (lg / 2))
        N = 8192 * 8192 // M
        x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 77 + lg)
        n8 = _l2_copies(dev, M * K + N * K + 2 * M * N)
        sets = [(A, B, torch.empty((M, N), dtype=torch.bfloat16, device=dev))] + \
               [(A.clone(), B.clone(), torch.empty((M, N), dtype=torch.bfloat16, device=dev))
                for _ in range(n8 - 1)]
        ms = _time_ms([lambda a=a, b=b, c=c: gb.gemm_fp8_dense(a, b, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=c)
                       for a, b, c in sets])
        del sets
        nb = _l2_copies(dev, 2 * M * K + 2 * N * K + 2 * M * N)
        bsets = [(x.bfloat16(), w.bfloat16()) for _ in range(nb)]
        ms_bf16 = _time_ms([lambda xb=xb, wb=wb: torch.matmul(xb, wb.T) for xb, wb in bsets])
        del bsets, x, w, A, B
        torch.cuda.empty_cache()
        flops = 2.0 * M * N * K
        rows.append({"M": M, "N": N, "K": K, "m_over_n": M / N, "fp8_ms": ms,
                     "fp8_tflops": flops / ms / 1e9, "bf16_ms": ms_bf16,
                     "bf16_tflops": flops / ms_bf16 / 1e9, "speedup_vs_bf16": ms_bf16 / ms,
                     "operand_copies": [n8, nb]})
    return rows


def format_sweep(gb, dev):
    """The four operand-format pairings (E4M3 / E5M2 for each operand, paper
    Table 3) on the same dense shapes, plus the quantisation rate of each
    format.  Operands rotate through copies as in the shape sweep."""
    rows = []
    for (M, N, K) in [(8192, 8192, 8192), (16384, 16384, 16384),
                      (16, workloads.SKINNY_NK, workloads.SKINNY_NK)]:
        for af in (0, 1):
            for bf in (0, 1):
                x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 5 * M + N, af, bf)
                del x, w
                n8 = _l2_copies(dev, M * K + N * K + 2 * M * N)
                sets = [(A, B, torch.empty((M, N), dtype=torch.bfloat16, device=dev))] + \
                       [(A.clone(), B.clone(), torch.empty((M, N), dtype=torch.bfloat16, device=dev))
                        for _ in range(n8 - 1)]
                ms = _time_ms([lambda a=a, b=b, c=c: gb.gemm_fp8_dense_fmt(
                    a, b, dA, 1, dB, 1, 1.0, gb.OUT_BF16, af, bf, C=c) for a, b, c in sets])
                del sets, A, B
                torch.cuda.empty_cache()
                rows.append({"M": M, "N": N, "K": K, "a_format": FORMAT_NAMES[af],
                             "b_format": FORMAT_NAMES[bf], "ms": ms,
                             "tflops": 2.0 * M * N * K / ms / 1e9, "operand_copies": n8})
    quant = []
    R = C = 8192
    x = torch.randn((R, C), device=dev)
    for fmt, fn in ((0, gb.fp8_quantize_e4m3), (1, gb.fp8_quantize_e5m2)):
        for mode in (0, 1):
            q = torch.empty((R, C), dtype=torch.uint8, device=dev)
            d = torch.empty((R if mode else 1,), dtype=torch.float32, device=dev)
            n = _l2_copies(dev, R * C * 5)
            xs = [x] + [x.clone() for _ in range(n - 1)]
            ms = _time_ms([lambda xx=xx: fn(xx, mode, q, d) for xx in xs])
            quant.append({"format": FORMAT_NAMES[fmt], "scale_mode": mode, "rows": R, "cols": C,
                          "us": ms * 1e3, "gbs": R * C * 5 / ms / 1e6, "input_copies": n})
            del xs
    return {"dense": rows, "quantize": quant}


def mx_sweep(gb, dev):
    """Block-scaled (MX, one E8M0 scale per 32 elements of K) against per-row
    scaled E4M3 on the same shapes: device time per call with L2-cold
    operand rotation, bf16 out."""
    rows = []
    for M, N, K in ((4096, 4096, 4096), (8192, 8192, 8192), (16384, 16384, 16384), (16, 8192, 8192),
                    (128, 8192, 8192), (2048, 2048, 2048)):
        n = _l2_copies(dev, M * K + N * K)
        mx_fns, row_fns, keep = [], [], []
        for i in range(n):
            g = torch.Generator(device=dev).manual_seed(100 + i)
            x = torch.randn((M, K), generator=g, device=dev)
            w = torch.randn((N, K), generator=g, device=dev)
            A, SA = gb.fp8_quantize_mx(x, gb.E4M3, scale_layout=1)
            B, SB = gb.fp8_quantize_mx(w, gb.E4M3, scale_layout=1)
            Ar, dA = gb.fp8_quantize_e4m3(x, 1)
            Br, dB = gb.fp8_quantize_e4m3(w, 1)
            del x, w
            C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
            keep += [A, SA, B, SB, Ar, dA, Br, dB, C]
            mx_fns.append(lambda A=A, SA=SA, B=B, SB=SB, C=C: gb.gemm_fp8_mx(A, SA, B, SB, 1.0, gb.OUT_BF16, C=C))
            row_fns.append(lambda A=Ar, dA=dA, B=Br, dB=dB, C=C: gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 1.0,
                                                                                    gb.OUT_BF16, C=C))
        ms_mx, ms_row = _time_ms(mx_fns), _time_ms(row_fns)
        f = 2.0 * M * N * K
        rows.append({"M": M, "N": N, "K": K, "mx_us": ms_mx * 1e3, "per_row_us": ms_row * 1e3,
                     "mx_tflops": f / ms_mx / 1e9, "per_row_tflops": f / ms_row / 1e9,
                     "mx_over_per_row": ms_row / ms_mx, "operand_copies": n})
        del keep, mx_fns, row_fns
    return rows


def mx_quant_sweep(gb, dev):
    """Quantisers alone: per-row E4M3 against block-scaled (tiled and
    row-major scale layouts), device time per call with L2-cold rotation;
    GB/s counts 4 bytes read and 1 written per element."""
    rows = []
    for R, C in ((4096, 4096), (8192, 8192), (16384, 8192)):
        n = _l2_copies(dev, R * C * 4)
        xs = [torch.randn((R, C), generator=torch.Generator(device=dev).manual_seed(300 + i), device=dev)
              for i in range(n)]
        q = torch.empty((R, C), dtype=torch.uint8, device=dev)
        d = torch.empty(R, device=dev)
        st = torch.empty(gb.fp8_mx_scale_tiled_bytes(R, C), dtype=torch.uint8, device=dev)
        sr = torch.empty((R, C // 32), dtype=torch.uint8, device=dev)
        ms_row = _time_ms([lambda x=x: gb.fp8_quantize_e4m3(x, 1, q, d) for x in xs])
        ms_t = _time_ms([lambda x=x: gb.fp8_quantize_mx(x, gb.E4M3, 1, q, st) for x in xs])
        ms_r = _time_ms([lambda x=x: gb.fp8_quantize_mx(x, gb.E4M3, 0, q, sr) for x in xs])
        b = R * C * 5
        rows.append({"rows": R, "cols": C, "per_row_us": ms_row * 1e3, "per_row_gbs": b / ms_row / 1e6,
                     "mx_tiled_us": ms_t * 1e3, "mx_tiled_gbs": b / ms_t / 1e6,
                     "mx_row_major_us": ms_r * 1e3, "mx_row_major_gbs": b / ms_r / 1e6, "copies": n})
        del xs
    return rows


def pair_sweep(gb, dev):
    """Dense GEMMs on CTA-pair tiles (mt 3, tcgen05 cta_group::2, 256 x 256
    per SM pair) against one-CTA 256-row tiles (mt 2) and 128-row tiles
    (mt 1): device time per call, L2-cold operand rotation, per-row scales,
    bf16 out; the transformer layer as one grouped launch."""
    rows = []
    shapes = [(2048, 2048, 2048), (4096, 4096, 4096), (8192, 8192, 8192), (16384, 16384, 16384),
              (2048, 8192, 8192), (8192, 2048, 8192), (4096, 14336, 4096)]
    for M, N, K in shapes:
        n = _l2_copies(dev, M * K + N * K)
        ops = []
        for i in range(n):
            x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 200 + i)
            del x, w
            ops.append((A, dA, B, dB, torch.empty((M, N), dtype=torch.bfloat16, device=dev)))
        fns = [lambda A=A, dA=dA, B=B, dB=dB, C=C: gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=C)
               for A, dA, B, dB, C in ops]
        row = {"M": M, "N": N, "K": K, "operand_copies": n}
        for mt in (1, 2, 3):
            gb.fp8_gemm_set_tile_config(mt, 0)
            row[f"mt{mt}_plan"] = gb.gemm_fp8_dense_plan(M, N, K)["mt"]
            ms = _time_ms(fns)
            row[f"mt{mt}_us"] = ms * 1e3
            row[f"mt{mt}_tflops"] = 2.0 * M * N * K / ms / 1e9
        gb.fp8_gemm_set_tile_config(0, 0)
        rows.append(row)
        del ops, fns
    # transformer layer, one grouped launch
    probs, keep = [], []
    flops = 0.0
    for i, (_, M, N, K) in enumerate(workloads.TRANSFORMER_LAYER):
        x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 300 + i)
        del x, w
        C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
        keep += [A, dA, B, dB, C]
        probs.append(gb.make_problem(A, B, dA, 1, dB, 1, C, 1.0, gb.OUT_BF16))
        flops += 2.0 * M * N * K
    layer = {"shape": "transformer layer, 4 GEMMs grouped"}
    for mt in (1, 2, 3):
        gb.fp8_gemm_set_tile_config(mt, 0)
        ms = _time_ms(lambda: gb.gemm_fp8_grouped(probs))
        layer[f"mt{mt}_ms"] = ms
        layer[f"mt{mt}_tflops"] = flops / ms / 1e9
    gb.fp8_gemm_set_tile_config(0, 0)
    del keep
    return {"gemms": rows, "layer": layer}


def prune_sweep(gb, dev):
    """prune24_compress alone: device time per call and HBM rate (1 byte
    read + 0.625 bytes written per element), L2-cold rotation."""
    rows = []
    for M, K in ((4096, 4096), (8192, 8192), (16384, 16384), (512, 1024)):
        n = _l2_copies(dev, M * K)
        ops = []
        for i in range(n):
            A = torch.randint(0, 256, (M, K), dtype=torch.uint8, device=dev)
            ops.append((A, torch.empty((M, K // 2), dtype=torch.uint8, device=dev),
                        torch.empty((M, K // 8), dtype=torch.uint8, device=dev)))
        fns = [lambda A=A, v=v, m=m: gb.prune24_compress(A, v, m) for A, v, m in ops]
        ms = _time_ms(fns)
        rows.append({"M": M, "K": K, "us": ms * 1e3, "gbs": M * K * 1.625 / ms / 1e6, "copies": n})
        del ops, fns
    return rows


def raster_sweep(gb, dev):
    """Raster band height (M-blocks per band) of the tile walk for CTA-pair
    tiles (mt 3) and one-CTA 256-row tiles (mt 2) on large squares: device
    time per call, L2-cold rotation."""
    rows = []
    for n_ in (8192, 16384):
        n = _l2_copies(dev, 2 * n_ * n_)
        ops = []
        for i in range(n):
            x, w, A, dA, B, dB = _operands(gb, n_, n_, n_, dev, 400 + i)
            del x, w
            ops.append((A, dA, B, dB, torch.empty((n_, n_), dtype=torch.bfloat16, device=dev)))
        fns = [lambda A=A, dA=dA, B=B, dB=dB, C=C: gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=C)
               for A, dA, B, dB, C in ops]
        for mt in (2, 3):
            for gm in (2, 4, 8, 12, 16, 32, 64):
                gb.fp8_gemm_set_tile_config(mt, gm)
                ms = _time_ms(fns)
                rows.append({"n": n_, "mt": mt, "group_m": gm, "us": ms * 1e3,
                             "tflops": 2.0 * n_ ** 3 / ms / 1e9})
        gb.fp8_gemm_set_tile_config(0, 0)
        del ops, fns
    return rows


def serving_policy_sweep(gb, dev, n=20000, load=0.8):
    """The batched server with the bulk tenant leaving R SMs free for the
    latency tenant, R in {0, 8, 16, 24, 32}, against per-call serving, on
    one seeded Poisson trace at `load` x the per-call capacity."""
    sb = ServingBench(dev, gb)
    sms = gb.fp8_device_sm_count()
    reqs = sb.trace(n, workloads.SEED_REQUESTS)
    tenant = np.array([r["tenant"] for r in reqs])
    sb.run(reqs[:256], dict(batching=False))
    _, span, _, _ = sb.run(reqs, dict(batching=False))
    rate = load * n / (span * 1e-6)
    out = {"offered_req_per_s": rate, "requests": n, "rows": []}
    share = dict(latency_pool_bytes=ServingBench.LATENCY_POOL)
    cfgs = [("per_call", dict(batching=False)),
            ("batched_reserve_16", dict(batching=True, bulk_max_ctas=sms - 16)),
            ("batched_reserve_16_latency_pool", dict(batching=True, bulk_max_ctas=sms - 16, **share)),
            ("batched_reserve_16_pool_32g", dict(batching=True, bulk_max_ctas=sms - 16, pool_bytes=32 << 30)),
            ("batched_reserve_0_latency_pool", dict(batching=True, **share)),
            ("batched_reserve_32_latency_pool", dict(batching=True, bulk_max_ctas=sms - 32, **share)),
            ("batched_waves_8x_latency_pool", dict(batching=True, bulk_max_ctas=8 * sms, **share))]
    traces = [reqs, sb.trace(n, workloads.SEED_REQUESTS + 7)]
    for name, cfg in cfgs:
        for k, tr in enumerate(traces):
            ten = np.array([r["tenant"] for r in tr])
            lat, span, stats, _ = sb.run(tr, cfg, rate)
            row = {"mode": name, "trace": k,
                   "p99_us": {f"tenant{t}": float(np.percentile(lat[ten == t], 99)) for t in (0, 1)},
                   "p50_us": {f"tenant{t}": float(np.percentile(lat[ten == t], 50)) for t in (0, 1)},
                   "p99_all_us": float(np.percentile(lat, 99)),
                   "pool_high_water_mb": stats["pool_high_water"] / 2 ** 20,
                   "max_batch": int(stats["max_batch_seen"]),
                   "submit_lag_us": stats["submit_lag_us"]}
            if k == 0:
                _, cspan, _, _ = sb.run(tr[:8000], cfg)
                row["capacity_req_per_s"] = 8000 / (cspan * 1e-6)
            out["rows"].append(row)
    return out


SWEEP_SECTIONS = ("shapes", "formats", "occupancy", "aspect", "serving", "concurrency", "mx", "mx_quant",
                  "serving_policy", "served_concurrency", "pair", "raster", "prune")


def sweep(gb, dev, sections=SWEEP_SECTIONS):
    """The measurement tables beyond the one-line step: `sections` picks
    from SWEEP_SECTIONS."""
    pk, _ = peaks()
    out = {}
    if "shapes" in sections:
        out.update(shape_sweep(gb, dev))
    if "formats" in sections:
        out["formats"] = format_sweep(gb, dev)
    if "occupancy" in sections:
        out["occupancy"] = occupancy_sweep(gb, dev, pk["bf16_tflops"] * FP8_PER_BF16)
    if "aspect" in sections:
        out["aspect_ratio"] = aspect_sweep(gb, dev)
    if "serving" in sections:
        out["serving"] = serving_report(gb, dev, loads=(0.8, 0.5, 0.95))
    if "concurrency" in sections:
        out["concurrency"] = concurrency_sweep(gb, dev)
    if "mx" in sections:
        out["mx"] = mx_sweep(gb, dev)
    if "mx_quant" in sections:
        out["mx_quant"] = mx_quant_sweep(gb, dev)
    if "serving_policy" in sections:
        out["serving_policy"] = serving_policy_sweep(gb, dev)
    if "served_concurrency" in sections:
        out["served_concurrency"] = served_concurrency_sweep(gb, dev)
    if "pair" in sections:
        out["pair"] = pair_sweep(gb, dev)
    if "raster" in sections:
        out["raster"] = raster_sweep(gb, dev)
    if "prune" in sections:
        out["prune"] = prune_sweep(gb, dev)
    return out


def shape_sweep(gb, dev):
    """Configs 2-4: dense square and skinny vs BF16 torch.matmul, 2:4 sparse
    vs dense on the same pruned A, the transformer layer as one grouped
    persistent launch vs per-call.  Every row rotates through copies of its
    operands (see _l2_copies) so no timed call finds them in L2; the
    transformer layer's operands are far larger than L2 already."""
    out = {"dense": [], "sparse": [], "transformer_layer": None}
    # config 1: the small dense case (per-tensor scales, FP32 out): a
    # latency point, one launch's fixed cost
    M, N, K = workloads.DENSE_SMALL
    g = torch.Generator(device=dev).manual_seed(workloads.SEED_A)
    x = torch.randn((M, K), generator=g, device=dev)
    w = torch.randn((N, K), generator=g, device=dev)
    A, dA = gb.fp8_quantize_e4m3(x, 0)
    B, dB = gb.fp8_quantize_e4m3(w, 0)
    n1 = _l2_copies(dev, M * K + N * K + 4 * M * N)
    sets = [(A.clone(), B.clone(), torch.empty((M, N), device=dev)) for _ in range(n1)]
    ms = _time_ms([lambda a=a, b=b, c=c: gb.gemm_fp8_dense(a, b, dA, 0, dB, 0, 1.0, gb.OUT_F32, C=c)
                   for a, b, c in sets])
    bsets = [(x.bfloat16(), w.bfloat16()) for _ in range(n1)]
    ms_bf16 = _time_ms([lambda xb=xb, wb=wb: torch.matmul(xb, wb.T) for xb, wb in bsets])
    out["dense_small"] = {"M": M, "N": N, "K": K, "scales": "per tensor", "out": "fp32",
                          "fp8_us": ms * 1e3, "bf16_matmul_us": ms_bf16 * 1e3,
                          "fp8_tflops": 2.0 * M * N * K / ms / 1e9}
    del sets, bsets
    for (M, N, K) in [(s, s, s) for s in workloads.SQUARE_SWEEP] + \
                     [(m, workloads.SKINNY_NK, workloads.SKINNY_NK) for m in workloads.SKINNY_M]:
        x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, M + N)
        n8 = _l2_copies(dev, M * K + N * K + 2 * M * N)
        sets = [(A, B, torch.empty((M, N), dtype=torch.bfloat16, device=dev))] + \
               [(A.clone(), B.clone(), torch.empty((M, N), dtype=torch.bfloat16, device=dev))
                for _ in range(n8 - 1)]
        ms = _time_ms([lambda a=a, b=b, c=c: gb.gemm_fp8_dense(a, b, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=c)
                       for a, b, c in sets])
        del sets
        nb = _l2_copies(dev, 2 * M * K + 2 * N * K + 2 * M * N)
        bsets = [(x.bfloat16(), w.bfloat16()) for _ in range(nb)]
        ms_bf16 = _time_ms([lambda xb=xb, wb=wb: torch.matmul(xb, wb.T) for xb, wb in bsets])
        del bsets
        flops = 2.0 * M * N * K
        row = {"M": M, "N": N, "K": K, "fp8_ms": ms, "fp8_tflops": flops / ms / 1e9,
               "bf16_matmul_ms": ms_bf16, "bf16_tflops": flops / ms_bf16 / 1e9,
               "speedup_vs_bf16": ms_bf16 / ms, "operand_copies": [n8, nb]}
        if M <= 128:
            row["fp8_gbs"] = (M * K + N * K + 2 * M * N) / ms / 1e6
        out["dense"].append(row)
        del x, w, A, B
        torch.cuda.empty_cache()
    sp_shapes = [(s, s, s) for s in workloads.SPARSE_SQUARE] + [workloads.SPARSE_SKINNY, workloads.SPARSE_RECT]
    for (M, N, K) in sp_shapes:
        x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 7 * M + N)
        vals, meta = gb.prune24_compress(A)
        Ap = gb.prune24_decompress(vals, meta, K)
        C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
        n8 = _l2_copies(dev, M * K + N * K + 2 * M * N)
        sp_sets = [(vals, meta, Ap, B, C)] + [(vals.clone(), meta.clone(), Ap.clone(), B.clone(), C.clone())
                                             for _ in range(n8 - 1)]
        ms_sp = _time_ms([lambda v=v, m=m, b=b, c=c: gb.gemm_fp8_sparse24(v, m, b, dA, 1, dB, 1, 1.0,
                                                                        gb.OUT_BF16, C=c)
                          for v, m, _, b, c in sp_sets])
        ms_d = _time_ms([lambda a=a, b=b, c=c: gb.gemm_fp8_dense(a, b, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=c)
                         for _, _, a, b, c in sp_sets])
        del sp_sets
        n_pr = _l2_copies(dev, M * K * 13 // 8)
        pr_sets = [(A, vals, meta)] + [(A.clone(), vals.clone(), meta.clone()) for _ in range(n_pr - 1)]
        ms_pr = _time_ms([lambda a=a, v=v, m=m: gb.prune24_compress(a, v, m) for a, v, m in pr_sets])
        del pr_sets
        flops = 2.0 * M * N * K
        row = {"M": M, "N": N, "K": K, "sparse_ms": ms_sp, "dense_same_pruned_ms": ms_d,
               "sparse_tflops_dense_equiv": flops / ms_sp / 1e9, "dense_tflops": flops / ms_d / 1e9,
               "sparse_speedup": ms_d / ms_sp, "prune_us": ms_pr * 1e3,
               "prune_gbs": M * K * 1.625 / ms_pr / 1e6}
        if M <= 512 and N > M:
            # sparse weights: the [N, K] operand pruned and put on the MMA M side
            wv, wm = gb.prune24_compress(B)
            Bp = gb.prune24_decompress(wv, wm, K)
            Ct = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
            w_sets = [(wv, wm, Bp)] + [(wv.clone(), wm.clone(), Bp.clone()) for _ in range(n8 - 1)]
            ms_ws = _time_ms([lambda v=v, m=m: gb.gemm_fp8_sparse24(v, m, A, dB, 1, dA, 1, 1.0, gb.OUT_BF16,
                                                                    out_transposed=True, C=Ct)
                              for v, m, _ in w_sets])
            ms_wd = _time_ms([lambda b=b: gb.gemm_fp8_dense(A, b, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=Ct)
                              for _, _, b in w_sets])
            del w_sets
            row.update({"weight_sparse_ms": ms_ws, "dense_same_pruned_weight_ms": ms_wd,
                        "weight_sparse_speedup": ms_wd / ms_ws})
        out["sparse"].append(row)
        del x, w, A, B, C, vals, meta, Ap
        torch.cuda.empty_cache()
    # transformer layer: QKV, output projection, FFN up, FFN down
    probs, keep, flops = [], [], 0.0
    calls_fp8, calls_bf16 = [], []
    for i, (name, M, N, K) in enumerate(workloads.TRANSFORMER_LAYER):
        x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 900 + i)
        C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
        xb, wb = x.bfloat16(), w.bfloat16()
        del x, w
        keep += [A, dA, B, dB, C, xb, wb]
        probs.append(gb.make_problem(A, B, dA, 1, dB, 1, C, 1.0, gb.OUT_BF16))
        calls_fp8.append((A, B, dA, dB, C))
        calls_bf16.append((xb, wb))
        flops += 2.0 * M * N * K
    tuned = gb.gemm_fp8_grouped_autotune(probs, iters=2)
    graph = gb.GroupedGraph(probs)
    ms_graph = _time_ms(graph.launch, capture=False)
    ms_grouped = _time_ms(lambda: gb.gemm_fp8_grouped(probs))
    ms_percall = _time_ms(lambda: [gb.gemm_fp8_dense(a, b, da, 1, db, 1, 1.0, gb.OUT_BF16, C=c)
                                   for a, b, da, db, c in calls_fp8])
    ms_bf16 = _time_ms(lambda: [torch.matmul(xb, wb.T) for xb, wb in calls_bf16])
    graph.close()
    out["transformer_layer"] = {
        "problems": [list(t) for t in workloads.TRANSFORMER_LAYER], "gflop": flops / 1e9,
        "tuned_tile": tuned,
        "grouped_graph_ms": ms_graph, "grouped_graph_tflops": flops / ms_graph / 1e9,
        "grouped_ms": ms_grouped, "fp8_per_call_ms": ms_percall,
        "bf16_per_call_ms": ms_bf16, "bf16_tflops": flops / ms_bf16 / 1e9,
        "speedup_vs_bf16_per_call": ms_bf16 / ms_graph}
    del keep
    torch.cuda.empty_cache()
    return out


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
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--tile", default=None,
                    help="mt[,group_m]: force the GEMM tile kind (1, 2, 3 = CTA pairs) and raster band")
    ap.add_argument("--sweep", default=None,
                    help="write the measurement tables to this JSON file and exit")
    ap.add_argument("--sections", default=",".join(SWEEP_SECTIONS),
                    help="comma list of sweep tables: " + ", ".join(SWEEP_SECTIONS))
    ap.add_argument("--gemm", default=None,
                    help="M,N,K[,sparse|mx][,mt1|mt2|mt3][,e4m3|e5m2,e4m3|e5m2]: run only this GEMM (warmup + "
                         "steps launches; for profilers); the two formats are A's and B's")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import paper_2602_10262_gb300 as gb
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    gb.library()
    if args.tile:
        t = [int(v) for v in args.tile.split(",")]
        gb.fp8_gemm_set_tile_config(t[0], t[1] if len(t) > 1 else 0)
    if args.gemm:
        f = args.gemm.split(",")
        M, N, K = (int(v) for v in f[:3])
        sparse = "sparse" in f[3:]
        mx = "mx" in f[3:]
        fmts = [{"e4m3": 0, "e5m2": 1}[t] for t in f[3:] if t in ("e4m3", "e5m2")] or [0, 0]
        af, bf = fmts[0], fmts[-1]
        x, w, A, dA, B, dB = _operands(gb, M, N, K, dev, 1, af, bf)
        C = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
        for t in f[3:]:
            if t.startswith("mt"):
                gb.fp8_gemm_set_tile_config(int(t[2:]), 0)
        if mx:
            A, SA = gb.fp8_quantize_mx(x, af, scale_layout=1)
            B, SB = gb.fp8_quantize_mx(w, bf, scale_layout=1)
            fn = lambda: gb.gemm_fp8_mx(A, SA, B, SB, 1.0, gb.OUT_BF16, af, bf, C=C)
        elif sparse:
            vals, meta = gb.prune24_compress(A)
            fn = lambda: gb.gemm_fp8_sparse24_fmt(vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16,
                                                  False, af, bf, C=C)
        else:
            fn = lambda: gb.gemm_fp8_dense_fmt(A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, af, bf, C=C)
        for _ in range(args.warmup + args.steps):
            fn()
        torch.cuda.synchronize()
        ms = _time_ms(fn)
        print(json.dumps({"gemm": args.gemm, "ms": ms, "tflops": 2.0 * M * N * K / ms / 1e9}))
        return 0
    if args.sweep:
        res = sweep(gb, dev, [t for t in args.sections.split(",") if t])
        pk, pk_kind = peaks()
        res["peaks"] = {"fp8_dense_tflops": pk["bf16_tflops"] * FP8_PER_BF16, "kind": pk_kind,
                        "hbm_gbs": pk["hbm_gbs"]}
        with open(args.sweep, "w") as f:
            json.dump(res, f, indent=1)
        print(json.dumps({"sweep": args.sweep}))
        return 0
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

    # does the loaded library run the sparse path?
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
    # fused quantise + 2:4 compress of A, quantise B, dense, 2:4 sparse; or,
    # without the sparse path: quantise A and B, compress A, dense
    launches_per_step = 4

    ev = {}

    def step(record=None):
        if record is not None:
            record[0].record(stream)
        if sparse_ok:
            # A's codes, scales and 2:4 compression in one pass over x
            gb.fp8_quantize_e4m3_prune24(x, A, dA, vals, meta)
        else:
            gb.fp8_quantize_e4m3(x, 1, A, dA)
        gb.fp8_quantize_e4m3(w, 1, B, dB)
        if not sparse_ok:
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
    with ClockSampler(local, gpu_uuid(dev)) as clocks:
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
    # the timed steps' own results on the oracle's sub-block, kept for the
    # parity check of the CPU leg below
    ca, cb = min(args.cpu_rows, M), min(args.cpu_cols, N)
    gpu_block = {"A": A[:ca].cpu().numpy(), "dA": dA[:ca].cpu().numpy(), "B": B[:cb].cpu().numpy(),
                 "dB": dB[:cb].cpu().numpy(), "vals": vals[:ca].cpu().numpy(), "meta": meta[:ca].cpu().numpy(),
                 "Cd": Cd[:ca, :cb].float().cpu().numpy(),
                 "Cs": Cs[:ca, :cb].float().cpu().numpy() if sparse_ok else None}

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
    # B (+ scales) and 0.625 B of kept codes and metadata per element of A
    # (written by the fused pass; a separate prune also reads A's codes again)
    prep_bytes = (2 * 5.0 + 0.625 + (0.0 if sparse_ok else 1.0)) * M * K
    stages["quantize_prune_gbs"] = prep_bytes / (t_prep * 1e-3) / 1e9

    # ---------------------------------------------------------------- e2e
    # Every step copies its inputs (fp32 A and B) from pinned host memory,
    # runs the pipeline through the C ABI and reads both bf16 results back.
    # Steps are pipelined the way a serving loop would run them: step i + 1's
    # inputs travel host -> device and step i - 1's results device -> host
    # while step i computes (double-buffered device inputs and outputs, one
    # stream each for copy-in, compute and copy-out).
    e2e = None
    if not args.no_e2e:
        xp = x_h.pin_memory()
        wp = w_h.pin_memory()
        outs_h = [[torch.empty((M, N), dtype=torch.bfloat16).pin_memory() for _ in range(2 if sparse_ok else 1)]
                  for _ in range(2)]
        xs = [x, torch.empty_like(x)]
        wsb = [w, torch.empty_like(w)]
        outs_d = [[Cd, Cs] if sparse_ok else [Cd], [torch.empty_like(Cd), torch.empty_like(Cs)] if sparse_ok
                  else [torch.empty_like(Cd)]]
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        s_comp = torch.cuda.Stream()
        n_e2e = max(4, min(args.steps, 12))

        def run_steps(n):
            ev_in = [None, None]        # inputs of buffer b landed
            ev_comp = [None, None]      # compute on buffer b done (inputs free, outputs ready)
            ev_out = [None, None]       # results of buffer b read back (outputs free)
            for i in range(n):
                b = i % 2
                with torch.cuda.stream(s_in):
                    if ev_comp[b] is not None:
                        s_in.wait_event(ev_comp[b])
                    xs[b].copy_(xp, non_blocking=True)
                    wsb[b].copy_(wp, non_blocking=True)
                    ev_in[b] = torch.cuda.Event()
                    ev_in[b].record(s_in)
                with torch.cuda.stream(s_comp):
                    s_comp.wait_event(ev_in[b])
                    if ev_out[b] is not None:
                        s_comp.wait_event(ev_out[b])
                    Co = outs_d[b]
                    if sparse_ok:
                        gb.fp8_quantize_e4m3_prune24(xs[b], A, dA, vals, meta)
                    else:
                        gb.fp8_quantize_e4m3(xs[b], 1, A, dA)
                        gb.prune24_compress(A, vals, meta)
                    gb.fp8_quantize_e4m3(wsb[b], 1, B, dB)
                    gb.gemm_fp8_dense(A, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=Co[0])
                    if sparse_ok:
                        gb.gemm_fp8_sparse24(vals, meta, B, dA, 1, dB, 1, 1.0, gb.OUT_BF16, C=Co[1])
                    ev_comp[b] = torch.cuda.Event()
                    ev_comp[b].record(s_comp)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev_comp[b])
                    for hbuf, dbuf in zip(outs_h[b], outs_d[b]):
                        hbuf.copy_(dbuf, non_blocking=True)
                    ev_out[b] = torch.cuda.Event()
                    ev_out[b].record(s_out)
            return ev_out[(n - 1) % 2]

        cur = torch.cuda.current_stream()
        run_steps(2)
        torch.cuda.synchronize()
        barrier(ws)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(cur)
        for st_ in (s_in, s_comp, s_out):
            st_.wait_event(s0)
        last = run_steps(n_e2e)
        cur.wait_event(last)
        s1.record(cur)
        torch.cuda.synchronize()
        barrier(ws)
        if gb.fp8_last_device_error() != 0:
            raise RuntimeError("device error during the end-to-end run")
        ms_e2e = max_over_ranks(s0.elapsed_time(s1), ws)
        h2d = (x_h.numel() + w_h.numel()) * 4
        d2h = M * N * 2 * (2 if sparse_ok else 1)
        e2e = {"value": flops_step * n_e2e * ws / (ms_e2e * 1e-3) / 1e12, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": ms_e2e / n_e2e, "steps": n_e2e,
               "path": "pinned host fp32 -> H2D -> C ABI (quantize, prune, dense, sparse) -> D2H bf16; "
                       "copies of neighbouring steps overlap compute (double-buffered, 3 streams)"}

    # ---------------------------------------------------------------- serving
    serving = None
    if not args.no_serving:
        del x_h, w_h
        serving = serving_report(gb, dev)

    # ---------------------------------------------------------------- CPU oracle
    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cores = cpu_cores()
        smp = OracleSample(S, args.cpu_rows, args.cpu_cols, cores)
        f, t = smp.run()
        cpu = {"value": f / t / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": smp.describe() + f", {t:.1f} s"}
        if sparse_ok:
            parity = smp.check(gpu_block)
        # the same oracle on one host thread, on a smaller block
        a1, b1 = max(1, args.cpu_rows // 32), max(1, args.cpu_cols // 16)
        smp.orc.set_threads(1)
        f1, t1 = smp.run(a1, b1)
        smp.orc.set_threads(cores)
        cpu["single_thread"] = {"value": f1 / t1 / 1e12, "unit": UNIT, "cores": 1,
                                "sample": f"A rows [0,{a1}) x B rows [0,{b1}) at K={S}, {t1:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "e4m3 (fp32 accumulate)",
            "data": "synthetic (seeded N(0,1) fp32, torch.Generator)",
            "config": config(S, ws),
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roofline, "stages": stages, "sparse_path": sparse_ok,
            "e2e": e2e, "cpu_baseline": cpu, "parity": parity, "clocks": clocks.summary(),
            "serving": serving,
        }
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
