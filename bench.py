#!/usr/bin/env python3
"""Benchmark of the exact digital circular convolution on GB300.

One step = one fused batched convolution (forward transforms of f and g,
pointwise product with N^-1, inverse transform) over the whole workload,
inputs resident in HBM.  Default workload: 4096 pairs, N = 2^14,
m = 13631489, 32-bit words (the uniform-batch configuration).  Prints ONE
JSON line on rank 0.  The default run also measures the other four
workloads (one small convolution, the large transforms, the uneven batch and
the serving mix) and attaches each under "configs"; --workload runs one of
them alone as the line's own workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload conv2|conv1|conv3|conv4|serve5|exact6|shift7] [--quick]

Multi-GPU (torchrun): every rank convolves its own batch (independent pairs,
no collective on the data path); the timing is the max over ranks and the
value counts the pairs of all ranks (weak scaling).

CPU baseline: the test oracle on the host cores -- its radix-2 convolution
(O(N log N)) on whole pairs of the workload, threaded over pairs and on one
thread, and its direct Eq. 1 (O(N^2)) on sampled outputs.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = 13631489
M64 = 70525124609
METRIC = "circular convolutions/sec and NTT GB/s vs HBM peak, batched vs plain form, bit-exact"
WORKLOADS = {
    # name: (batch, log2N, description)
    "conv2": (4096, 14, "uniform batch: 4096 pairs x N=2^14, m=13631489, uint32"),
    "conv1": (1, 10, "single convolution: 1 pair x N=2^10, m=13631489, uint32"),
    "conv3": (64, 19, "large transforms: 64 pairs x N=2^19, m=13631489, uint32, split column/row path"),
    "serve5": (None, None, "serving: Poisson arrivals at 20000 req/s of convolutions with N = 2^k, k uniform on "
                           "{8..18}, m=70525124609 (factor of F_19), uint64, continuous batching, pool-admitted"),
    "conv4": (10000, None, "uneven batch: 10000 pairs, N = 2^k with k uniform on {6..19}, m=13631489, uint32, "
                           "one batch plan replayed as a CUDA graph"),
    "shift7": (1 << 21, 6, "strict bit-shift transform: 2^21 pairs x N=64, m=641 (a factor of F_5), twiddles "
                           "as shifts modulo F_5, against the same kernel with Shoup products and the main path"),
    "exact6": (8192, 12, "exact integer filtering: 8192 pairs x N=2^12 of signed 16-bit samples and taps "
                         "(|h| <= 2^42), int64 in and out, Chinese remainder theorem over Rader primes"),
}
SUB_CONFIGS = ("conv1", "conv3", "conv4", "serve5")
IMAD_PER_SM_CLK = 64          # 32-bit IMAD lanes per SM per clock (GB300: 18.98 T IMAD/s measured over 152 SMs)
SLOTS_PER_MODMUL = 4          # Shoup product: IMAD.HI (2 issue slots of the IMAD pipe) + 2 IMAD
SCHEDULE = os.path.join(ROOT, "paper_1005_1497_gb300", "schedules", "gb300.json")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="conv2", choices=sorted(WORKLOADS))
    ap.add_argument("--quick", action="store_true",
                    help="fused timing only (no plain form, e2e, CPU baseline or other workloads)")
    ap.add_argument("--no-configs", action="store_true", help="do not measure the other workloads")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU oracle samples")
    ap.add_argument("--log2n", type=int, default=None,
                    help="override log2 N of the uniform workloads (conv1/conv2/conv3 shapes), e.g. for profiling")
    ap.add_argument("--batch", type=int, default=None,
                    help="override the number of pairs of the uniform workloads and of the uneven batch")
    ap.add_argument("--m64", action="store_true",
                    help="uniform workloads modulo the 64-bit-word prime 70525124609 (uint64), e.g. for profiling")
    ap.add_argument("--schedule", default=None,
                    help="schedule file to load (default: the packaged GB300 schedule when present, else the plans' "
                         "heuristics); with --tune, the file the tuned schedule is written to")
    ap.add_argument("--tune", action="store_true", help="autotune the split-path classes in this run instead")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ helpers

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    """Largest value over all ranks (the step time of the slowest GPU)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_pairs(total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous share [start, end) of `total` independent pairs for `rank`
    (used when a fixed job is split across GPUs; the benchmark itself gives
    every rank its own batch of the same size, i.e. weak scaling)."""
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def traffic_from_profile(kernel_tag: str):
    """DRAM bytes per launch recorded by an ncu capture summary in profiles/, if
    it was taken on the current kernel code (its kernel_digest line matches:
    the kernel-defining sources without comments, and the compile flags)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.txt")
    if not os.path.exists(path):
        return None
    from paper_1005_1497_gb300 import build
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line:
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_digest") != build.kernel_digest():
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def uniform_shape(name: str, args):
    """(batch, log2 N, description) of a uniform workload, with the overrides."""
    batch, L, desc = WORKLOADS[name]
    if name in ("conv1", "conv2", "conv3") and (args.log2n is not None or args.batch is not None or args.m64):
        L = args.log2n if args.log2n is not None else L
        batch = args.batch if args.batch is not None else batch
        word = "m=70525124609, uint64" if args.m64 else "m=13631489, uint32"
        desc = f"uniform batch: {batch} pairs x N=2^{L}, {word} (override)"
    return batch, L, desc


def config_of(name: str, args, world: int = 1) -> dict:
    """The workload's `config` object; both arms print the same one."""
    par = f"replicas x{world} (independent pairs per GPU)"
    if name in ("conv1", "conv2", "conv3"):
        batch, L, desc = uniform_shape(name, args)
        big = 8 * batch * (1 << L) > (129 << 20)
        return {"workload": desc, "batch_per_gpu": batch, "N": 1 << L, "m": M64 if args.m64 else M,
                "l2": "inputs larger than L2; no flush" if big else
                      "inputs smaller than L2: every step rereads them from L2 (no flush)",
                "parallelism": par}
    if name == "conv4":
        return {"workload": WORKLOADS[name][2] if args.batch is None else
                f"uneven batch: {args.batch} pairs, N = 2^k with k uniform on {{6..19}}, m=13631489, uint32 (override)",
                "pairs": args.batch or WORKLOADS[name][0], "m": M,
                "l2": "inputs larger than L2 (6 GB of f+g); no flush", "parallelism": par}
    if name == "serve5":
        return {"workload": WORKLOADS[name][2], "offered_req_per_s": 20000.0, "m": M64, "parallelism": par}
    batch, L, desc = WORKLOADS[name]
    if name == "exact6":
        return {"workload": desc, "batch_per_gpu": batch, "N": 1 << L,
                "l2": "inputs larger than L2 (512 MiB of int64 f+g); no flush", "parallelism": par}
    return {"workload": desc, "batch_per_gpu": batch, "N": 1 << L, "m": 641,
            "l2": "inputs larger than L2 (1 GiB of f+g); no flush", "parallelism": par}


def load_schedule(args, ntt) -> dict:
    """The autotuned schedules (split-path wave and form, whole-sequence
    threads per block, persistent-launch membership): the file given, or the
    packaged GB300 one, when it exists; none (the plans' heuristics) otherwise."""
    path = args.schedule if args.schedule else SCHEDULE
    if path and os.path.exists(path):
        ntt.ntt_autotune_load(path)
        return {"loaded": os.path.relpath(path, ROOT)}
    return {"loaded": None}


def alu_peak_gmodmul(local: int, sm_max_mhz: float) -> float:
    import torch
    return torch.cuda.get_device_properties(local).multi_processor_count * IMAD_PER_SM_CLK * sm_max_mhz * 1e6 \
        / SLOTS_PER_MODMUL / 1e9


# --------------------------------------------------------------- CPU oracle

def oracle_rate_mixed(pairs, budget_s: float, kind: str = "direct", threads: int | None = None):
    """Time the oracle on a list of pairs (f, g, m, kind_of_pair) on the host
    cores and return (conv/s, threads, work done, wall s).

    kind "direct": Eq. 1 on sampled outputs -- the modular or_conv_sample
    ("mod" pairs) or the exact integer or_int_conv_sample ("int" pairs).
    Every thread takes blocks of output indices round-robin over the pairs
    (8 on the first visit of a pair, 256 after); a pair's time is its sampled
    seconds scaled by N / outputs (each output costs N products).  Work done
    counts outputs.

    kind "fast": the oracle's radix-2 convolution (or_fast_conv) on whole
    pairs, round-robin, each pair at least once; a pair's time is the mean of
    its runs.  Work done counts whole pairs.  ("int" pairs have no fast form
    and are timed direct.)

    Either way the rate is threads x pairs over the sum of the pairs' times,
    which weighs every length of a mixed workload by its share of it."""
    import numpy as np

    import oracle
    o = oracle.Oracle()
    threads = threads or os.cpu_count() or 1
    P = len(pairs)
    stop = time.perf_counter() + budget_s
    lock = threading.Lock()
    nxt = [0]
    cursor, spent, units = [0] * P, [0.0] * P, [0] * P
    roots = {}

    def worker():
        while True:
            with lock:
                k = nxt[0]
                if k >= P and time.perf_counter() >= stop:
                    return
                nxt[0] += 1
                i = k % P
                f, g, m, pk = pairs[i]
                N = f.shape[-1]
                fast = kind == "fast" and pk == "mod"
                cnt = N if fast else min(N, 8 if k < P else 256)
                off = cursor[i]
                cursor[i] = (off + cnt) % N
                if fast and (m, N) not in roots:
                    roots[(m, N)] = o.root(m, N)
                w = roots.get((m, N))
            t = time.perf_counter()
            if fast:
                o.fast_conv(f, g, m, w)
            else:
                idx = ((off + np.arange(cnt, dtype=np.uint64)) % np.uint64(N)).astype(np.uint64)
                if pk == "int":
                    o.int_conv_sample(f, g, idx)
                else:
                    o.conv_sample(f, g, m, idx)
            dt = time.perf_counter() - t
            with lock:
                spent[i] += dt
                units[i] += cnt

    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    el = time.perf_counter() - t0
    est = sum(spent[i] * pairs[i][0].shape[-1] / units[i] for i in range(P))
    done = sum(units) if kind != "fast" else sum(u // pairs[i][0].shape[-1] for i, u in enumerate(units))
    return threads * P / est, threads, done, el


def reference_pairs(name: str, args, cap: int = 64):
    """Up to `cap` pairs of the workload, from the same seeded generators, in
    the workload's own length mix.  Returns (pairs, unit)."""
    import numpy as np

    from paper_1005_1497_gb300 import inputs
    if name == "conv4":
        lens = inputs.log_uniform_lengths(args.batch or WORKLOADS["conv4"][0], 6, 19, seed=1000)[:cap]
        return [(*(a[0] for a in inputs.pairs(M, 1, int(n), seed=1000 + i)), M, "mod")
                for i, n in enumerate(lens)], "conv/s"
    if name == "serve5":
        lens = inputs.log_uniform_lengths(512, 8, 18, seed=2000)[:cap]
        return [(*(a[0] for a in inputs.pairs(M64, 1, int(n), seed=2000 + i, dtype=np.uint64)), M64, "mod")
                for i, n in enumerate(lens)], "req/s"
    if name == "exact6":
        batch, L, _ = WORKLOADS[name]
        N, amp = 1 << L, 1 << 15
        out = []
        for i in range(min(batch, cap)):
            f = inputs.uniform_mod(2 * amp + 1, N, 1000 + i, 0, dtype=np.uint64).astype(np.int64) - amp
            g = inputs.uniform_mod(2 * amp + 1, N, 1000 + i, 1, dtype=np.uint64).astype(np.int64) - amp
            out.append((f, g, 0, "int"))
        return out, "conv/s"
    if name == "shift7":
        batch, L, _ = WORKLOADS[name]
        f, g = inputs.pairs(641, min(batch, cap), 1 << L, seed=1000)
        return [(f[i], g[i], 641, "mod") for i in range(f.shape[0])], "conv/s"
    batch, L, _ = uniform_shape(name, args)
    m = M64 if args.m64 else M
    f, g = inputs.pairs(m, min(batch, cap), 1 << L, seed=1000, dtype=np.uint64)
    return [(f[i], g[i], m, "mod") for i in range(f.shape[0])], "conv/s"


def cpu_baseline(name: str, args, budget_s: float, full: bool) -> dict:
    """The oracle's rates on the workload's own pairs (rank 0 at N=1 only):
    the radix-2 convolution threaded over pairs (the value), and with `full`
    the same on one thread and the direct Eq. 1 on sampled outputs."""
    pairs, unit = reference_pairs(name, args)
    integer = pairs[0][3] == "int"
    share = budget_s / (3 if full else 1)
    rate, thr, done, el = oracle_rate_mixed(pairs, share, kind="fast")
    what = ("exact integer Eq. 1 in 128-bit integers (oracle or_int_conv_sample), sampled outputs" if integer else
            "radix-2 Cooley-Tukey convolution of the oracle (or_fast_conv) on whole pairs, threads over pairs")
    out = {"value": round(rate, 4), "unit": unit, "cores": thr, "kind": "oracle",
           "sample": f"{what}: {done} {'outputs' if integer else 'pair convolutions'} over {len(pairs)} pairs of the "
                     f"workload in {el:.1f} s; rate = threads x pairs / sum of each pair's time"}
    if full and not integer:
        r1, _, d1, e1 = oracle_rate_mixed(pairs, share, kind="fast", threads=1)
        out["single_thread"] = {"value": round(r1, 4), "cores": 1, "pairs_done": d1, "seconds": round(e1, 1)}
        rd, thd, dd, ed = oracle_rate_mixed(pairs, share, kind="direct")
        out["direct"] = {"value": round(rd, 4), "cores": thd,
                         "sample": f"direct Eq. 1 (oracle or_conv_sample, O(N^2)) on {dd} sampled output indices "
                                   f"of {len(pairs)} pairs in {ed:.1f} s, each pair's time scaled to all N outputs"}
    return out


# ---------------------------------------------------------------- our path

def count_launches(ntt, fn) -> int:
    """Kernel launches one call of fn issues, by the library's own counter
    (an untimed call, before the warm-up)."""
    import torch
    c0 = ntt.launch_count()
    fn()
    torch.cuda.synchronize()
    return ntt.launch_count() - c0


def measure_uniform(name, args, world, rank, local, sub=False):
    """Uniform batches (conv1, conv2, conv3): one conv_circular per step."""
    import numpy as np
    import torch

    from paper_1005_1497_gb300 import inputs, ntt

    batch, L, desc = uniform_shape(name, args)
    N = 1 << L
    m = M64 if args.m64 else M
    wb = 8 if args.m64 else 4                                     # bytes per word
    tdt = torch.int64 if args.m64 else torch.int32
    schedule = {}
    if L > (13 if args.m64 else 14):                              # split path: form and pairs per wave
        if args.tune and not sub:
            t = ntt.ntt_autotune(m, N, batch)
            schedule = {"tuned": {k: t[k] for k in ("wave", "twist", "default_wave", "default_twist")},
                        "tuned_ms": round(t["ms"], 4), "heuristic_ms": round(t["default_ms"], 4)}
            if args.schedule:
                ntt.ntt_autotune_save(args.schedule)
    plan = ntt.Plan(m, N)
    if plan.four_step:
        schedule.update({"pairs_per_wave": plan.wave, "twist_form": plan.twist})
    else:
        schedule.update({"threads_per_block": plan.block})
    # inputs from the shared seeded generator (computed on the device), resident in HBM
    seed = 1000 + rank
    f = inputs.uniform_mod_torch(m, batch * N, seed, 0, device="cuda", dtype=tdt).view(batch, N)
    g = inputs.uniform_mod_torch(m, batch * N, seed, 1, device="cuda", dtype=tdt).view(batch, N)
    h = torch.empty_like(f)
    stream = torch.cuda.current_stream()

    def step():
        ntt.conv_circular(plan, f, g, out=h, stream=stream)

    launches_per_step = count_launches(ntt, step)

    # A launch-bound step (one small convolution) is replayed from a CUDA
    # graph captured once, so that the host's per-call cost is not timed as
    # GPU time; the plain launch is timed beside it.
    graph = None
    if batch * N <= (1 << 16):
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        cap = torch.cuda.Stream()
        cap.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(cap):
            with torch.cuda.graph(graph, stream=cap):
                ntt.conv_circular(plan, f, g, out=h, stream=cap)
        torch.cuda.synchronize()
    run = graph.replay if graph is not None else step
    # (a workload under `configs` times its own step count, stated in its line: a
    # graph-replayed step of a few microseconds is timed over 2000 replays)
    if not sub:
        steps = args.steps
    elif graph is not None:
        steps = max(args.steps, 2000)
    else:
        steps = max(1, min(args.steps, 400 if L > 14 else 2000))
    for _ in range(max(args.warmup, 3 if sub else 0)):
        run()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(steps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1) / steps
    plain_launch_ms = None
    if graph is not None:
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(steps):
            step()
        p1.record(stream)
        torch.cuda.synchronize()
        plain_launch_ms = p0.elapsed_time(p1) / steps
    ms = max_over_ranks(world, ms)
    clocks = clk.summary()
    pairs_total = batch * world
    value = pairs_total * 1000.0 / ms

    # roofline: the fused kernel (one launch per step when N fits one block),
    # or the split path's three kernels per wave, rows dominating
    hbm_peak, sm_max_mhz, peak_src = peaks()
    alg_bytes = 3.0 * wb * N * batch                              # f, g in, h out
    modmul = batch * (3 * (N // 2) * L + N)                      # butterfly products + pointwise
    launch_ms = ms / launches_per_step
    alu_peak = alu_peak_gmodmul(local, sm_max_mhz)
    alu_ach = modmul / (ms * 1e-3) / 1e9
    hbm_ach = alg_bytes / (ms * 1e-3) / 1e9
    if plan.four_step:
        kernel_tag = None
        kernel = ("split path, per wave k_cols_fwd + k_conv_cr<u32,14,14,0,1> (rows: 2^(L-14) whole length-2^14 "
                  "convolutions per pair, the dominant kernel) + k_cols_inv")
    elif L > (9 if args.m64 else 10):
        kernel_tag = None if args.m64 else f"k_conv_cr_u32_L{L}_{batch}x{N}"
        kernel = f"k_conv_cr<u{8 * wb},{L},{L},0,0,{plan.block}> (fused, column/row form)"
    elif batch <= plan.small_max:
        kernel_tag = None
        kernel = f"k_conv_small<u{8 * wb},{L}> (fused, one thread block per pair: a batch too small to fill the GPU)"
    else:
        kernel_tag = None
        kernel = f"k_conv_fused<u{8 * wb},{L},0,{plan.block}> (fused, one warp per sequence)"
    traffic = traffic_from_profile(kernel_tag) if kernel_tag else None
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "conv/s", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": f"u{8 * wb}", "data": "synthetic (seeded counter-based uniform residues in [0,m))",
        "config": config_of(name, args, world),
        "roofline": {"bound": "alu", "achieved": round(alu_ach, 1), "peak": round(alu_peak, 1), "unit": "Gmodmul/s",
                     "frac": round(alu_ach / alu_peak, 4), "traffic": traffic,
                     "peak_src": f"{IMAD_PER_SM_CLK} IMAD/clk/SM x SMs x {sm_max_mhz:.0f} MHz / {SLOTS_PER_MODMUL} "
                                 f"slots per Shoup product",
                     "kernel": kernel, "launch_ms": round(launch_ms, 4), "launches_per_step": launches_per_step},
        "roofline_hbm": {"bound": "hbm", "achieved": round(hbm_ach, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(hbm_ach / hbm_peak, 4), "peak_src": f"{peak_src} copy bandwidth",
                         "algorithmic_bytes_per_step": alg_bytes},
        "clocks": clocks,
        "gpu_launches": launches_per_step * steps,
    }
    if schedule:
        out["schedule"] = schedule
    if graph is not None:
        out["launch"] = {"timed": "CUDA graph replay of one conv_circular call per step",
                         "ms_per_step_plain_launch": round(plain_launch_ms, 4)}

    if not args.quick and not sub:
        # standalone natural-order transforms of the same batch (Eq. 2 and 3):
        # 8 algorithmic bytes per element (read x, write X)
        X = torch.empty_like(f)
        tsteps = max(1, min(args.steps // 4, 200))
        ntt_rates = {}
        for tname, fn in (("forward", ntt.ntt_forward), ("inverse", ntt.ntt_inverse)):
            for _ in range(3):
                fn(plan, f, out=X, stream=stream)
            torch.cuda.synchronize()
            t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0e.record(stream)
            for _ in range(tsteps):
                fn(plan, f, out=X, stream=stream)
            t1e.record(stream)
            torch.cuda.synchronize()
            tms = max_over_ranks(world, t0e.elapsed_time(t1e) / tsteps)
            gbps = 8.0 * N * batch / (tms * 1e-3) / 1e9
            ntt_rates[tname] = {"ms": round(tms, 4), "GBps": round(gbps, 1), "frac_hbm": round(gbps / hbm_peak, 4),
                                "transforms_per_s": round(batch * world * 1000.0 / tms, 1)}
        out["ntt"] = ntt_rates
        del X

        # plain form: one launch per butterfly stage over the whole batch
        work = torch.empty((2 * batch, N), dtype=tdt, device="cuda")
        h2 = torch.empty_like(f)
        for _ in range(max(args.warmup, 1)):
            ntt.conv_circular_plain(plan, f, g, out=h2, work=work, stream=stream)
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        psteps = max(1, min(args.steps // 2, 100))
        p0.record(stream)
        for _ in range(psteps):
            ntt.conv_circular_plain(plan, f, g, out=h2, work=work, stream=stream)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = max_over_ranks(world, p0.elapsed_time(p1) / psteps)
        same = bool(torch.equal(h, h2))
        out["plain_form"] = {"value": round(pairs_total * 1000.0 / pms, 1), "unit": "conv/s",
                             "ms_per_step": round(pms, 4), "launches_per_step": 2 * L + 2,
                             "algorithmic_GBps": round(alg_bytes / (pms * 1e-3) / 1e9, 1),
                             "fused_speedup": round(pms / ms, 2), "bit_identical_to_fused": same}
        del work, h2

    if not args.quick:
        # end to end through the host-buffer entry point (pinned host memory)
        fh = f.cpu().pin_memory()
        gh = g.cpu().pin_memory()
        hh = torch.empty_like(fh).pin_memory()
        for _ in range(max(args.warmup, 3)):               # (the host link's first steps run slow)
            ntt.conv_circular_host(plan, fh, gh, hh, stream=stream)
        esteps = max(1, min(args.steps, 20))
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(esteps):
            ntt.conv_circular_host(plan, fh, gh, hh, stream=stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(world, (time.perf_counter() - t0) * 1000.0 / esteps)
        out["e2e"] = {"value": round(pairs_total * 1000.0 / ems, 1), "unit": "conv/s", "ms_per_step": round(ems, 3),
                      "h2d_bytes_per_step": 2 * batch * N * wb, "d2h_bytes_per_step": batch * N * wb,
                      "entry": ("conv_circular_host (pinned host buffers: " + ("read and written in place by the kernel" if 3 * batch * N * wb <= (96 << 20) and not plan.four_step else "chunked copy/compute overlap") + ")"),
                      "bit_identical_to_device_path": bool(torch.equal(hh, h.cpu()))}
        # the host link alone, for the same bytes (plain copies, untimed
        # above): f and g in, h out, and both directions at once -- the
        # least time a step's copies can take
        side = torch.cuda.Stream()

        def copies_ms(h2d, d2h, reps=5):
            def once():
                if d2h:
                    side.wait_stream(torch.cuda.current_stream())
                    with torch.cuda.stream(side):
                        hh.copy_(h, non_blocking=True)
                if h2d:
                    f.copy_(fh, non_blocking=True)
                    g.copy_(gh, non_blocking=True)
                if d2h:
                    torch.cuda.current_stream().wait_stream(side)
            once()
            torch.cuda.synchronize()
            t = time.perf_counter()
            for _ in range(reps):
                once()
            torch.cuda.synchronize()
            return (time.perf_counter() - t) * 1000.0 / reps

        if 3 * batch * N * wb >= (64 << 20):     # (a few KB per step measure launch latency, not the link)
            in_ms, out_ms, both_ms = copies_ms(True, False), copies_ms(False, True), copies_ms(True, True)
            out["e2e"]["host_link"] = {"h2d_GBps": round(2 * batch * N * wb / (in_ms * 1e-3) / 1e9, 1),
                                       "d2h_GBps": round(batch * N * wb / (out_ms * 1e-3) / 1e9, 1),
                                       "both_directions_ms": round(both_ms, 3),
                                       "frac": round(both_ms / ems, 4),
                                       "note": "frac = the step's copies alone (both directions at once) / e2e step time"}
        if sub and plan.four_step:
            out["noalloc"] = noalloc_ratio(ntt, plan, f, g, h, stream, min(steps, 50))
        attach_cpu_baseline(out, name, args, world, rank, full=not sub)
    return out


def noalloc_ratio(ntt, plan, f, g, h, stream, steps) -> dict:
    """conv_circular_noalloc (split-path scratch in the library's fixed 16 MiB
    array, so small waves) against conv_circular on the same batch."""
    import ctypes

    import torch
    lib = ntt.lib()
    out = torch.empty_like(h)

    def call():
        st = lib.conv_circular_noalloc(plan.handle, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), f.shape[0], ctypes.c_void_p(stream.cuda_stream))
        if st != 0:
            raise RuntimeError(lib.ntt_last_error().decode())

    call()
    torch.cuda.synchronize()
    same = bool(torch.equal(out, h))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    na = e0.elapsed_time(e1) / steps
    e0.record(stream)
    for _ in range(steps):
        ntt.conv_circular(plan, f, g, out=h, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    wave = (16 << 20) // (2 * plan.N * (plan.word_bits // 8))
    return {"ms_per_step": round(na, 4), "conv_circular_ms": round(ms, 4), "ratio": round(na / ms, 3),
            "pairs_per_wave": wave, "bit_identical": same}


def measure_shift(args, world, rank, local, sub=False):
    """The strict bit-shift form (twiddles 2^e, e < 32, applied modulo F_5 =
    2^32 + 1 by shift and lo - hi; m = 641 divides F_5) against the same
    kernel with Shoup products modulo m and against the main fused path."""
    import torch

    from paper_1005_1497_gb300 import inputs, ntt

    batch, L, desc = WORKLOADS["shift7"]
    N, m = 1 << L, 641
    seed = 1000 + rank
    f = inputs.uniform_mod_torch(m, batch * N, seed, 0, device="cuda").view(batch, N)
    g = inputs.uniform_mod_torch(m, batch * N, seed, 1, device="cuda").view(batch, N)
    h = torch.empty_like(f)
    stream = torch.cuda.current_stream()
    plan = ntt.Plan(m, N)

    def timed(fn, steps):
        for _ in range(max(args.warmup, 1)):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(world, e0.elapsed_time(e1) / steps)

    steps = max(1, min(args.steps, 500))
    with ClockSampler(local) as clk:
        ms = timed(lambda: ntt.conv_circular_shift(m, f, g, out=h, mode=ntt.SHIFT_STRICT, stream=stream), steps)
    ref = h.clone()
    ms_shoup = timed(lambda: ntt.conv_circular_shift(m, f, g, out=h, mode=ntt.SHIFT_SHOUP, stream=stream), steps)
    same_shoup = bool(torch.equal(h, ref))
    ms_main = timed(lambda: ntt.conv_circular(plan, f, g, out=h, stream=stream), steps)
    same_main = bool(torch.equal(h, ref))
    hbm_peak, sm_max_mhz, peak_src = peaks()
    alg_bytes = 12.0 * N * batch
    hbm_ach = alg_bytes / (ms * 1e-3) / 1e9
    rate = lambda t: round(batch * world * 1000.0 / t, 1)
    out = {"metric": METRIC, "value": rate(ms), "unit": "conv/s", "n_gpus": world, "steps": steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64 lanes modulo F_5 (u32 in and out)",
           "data": "synthetic (seeded counter-based uniform residues in [0,641))",
           "config": config_of("shift7", args, world),
           "roofline": {"bound": "hbm", "achieved": round(hbm_ach, 1), "peak": hbm_peak, "unit": "GB/s",
                        "frac": round(hbm_ach / hbm_peak, 4), "traffic": None, "peak_src": f"{peak_src} copy bandwidth",
                        "kernel": "k_conv_shift<32, 6, strict>", "algorithmic_bytes_per_step": alg_bytes},
           "compare": {"same_kernel_shoup_products": {"value": rate(ms_shoup), "ms_per_step": round(ms_shoup, 4),
                                                      "bit_identical": same_shoup},
                       "main_fused_path": {"value": rate(ms_main), "ms_per_step": round(ms_main, 4),
                                           "bit_identical": same_main}},
           "clocks": clk.summary(), "gpu_launches": steps}
    # end to end: f and g copied in from pinned host memory, the strict
    # kernel, h copied back, every step
    fh, gh = f.cpu().pin_memory(), g.cpu().pin_memory()
    hh = torch.empty_like(fh).pin_memory()
    esteps = max(1, min(args.steps, 20))
    ew = max(args.warmup, 3)
    for i in range(esteps + ew):
        if i == ew:
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
        f.copy_(fh, non_blocking=True)
        g.copy_(gh, non_blocking=True)
        ntt.conv_circular_shift(m, f, g, out=h, mode=ntt.SHIFT_STRICT, stream=stream)
        hh.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    ems = max_over_ranks(world, (time.perf_counter() - t0) * 1000.0 / esteps)
    out["e2e"] = {"value": rate(ems), "unit": "conv/s", "ms_per_step": round(ems, 3),
                  "h2d_bytes_per_step": 8 * batch * N, "d2h_bytes_per_step": 4 * batch * N,
                  "entry": "conv_circular_shift (strict) between one host-to-device copy of f and of g (pinned) "
                           "and one device-to-host copy of h",
                  "bit_identical_to_device_path": bool(torch.equal(hh, ref.cpu()))}
    attach_cpu_baseline(out, "shift7", args, world, rank, full=False)
    return out


def measure_exact(args, world, rank, local, sub=False):
    """Exact (non-modular) convolution of signed 16-bit data: residues modulo
    each prime of the plan, one fused modular convolution per prime, Garner
    reconstruction to int64."""
    import torch

    from paper_1005_1497_gb300 import inputs, ntt

    batch, L, desc = WORKLOADS["exact6"]
    N = 1 << L
    amp = 1 << 15                                   # samples and taps in [-2^15, 2^15]
    bound = L + 31                                  # N amp^2 = 2^42 < 2^43
    plan = ntt.ExactPlan(N, bound)
    seed = 1000 + rank
    f = inputs.uniform_mod_torch(2 * amp + 1, batch * N, seed, 0, device="cuda", dtype=torch.int64).view(batch, N) - amp
    g = inputs.uniform_mod_torch(2 * amp + 1, batch * N, seed, 1, device="cuda", dtype=torch.int64).view(batch, N) - amp
    h = torch.empty_like(f)
    stream = torch.cuda.current_stream()

    def step():
        ntt.conv_exact(plan, f, g, out=h, stream=stream)

    launches_per_step = count_launches(ntt, step)         # per wave: residues, one conv per prime, reconstruction

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    steps = max(1, min(args.steps, 500))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(world, e0.elapsed_time(e1) / steps)
    hbm_peak, sm_max_mhz, peak_src = peaks()
    alg_bytes = 24.0 * N * batch                                   # int64 f, g in, h out
    modmul = batch * len(plan.primes) * (3 * (N // 2) * L + N)    # per prime: butterflies + pointwise
    alu_peak = alu_peak_gmodmul(local, sm_max_mhz)
    alu_ach = modmul / (ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": round(batch * world * 1000.0 / ms, 1), "unit": "conv/s", "n_gpus": world,
           "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64 (residues u32)",
           "data": "synthetic (seeded counter-based, uniform in [-2^15, 2^15])",
           "config": config_of("exact6", args, world),
           "plan": {"bound_bits": bound, "primes": plan.primes, "word_bits": plan.word_bits, "pairs_per_wave": plan.wave},
           "roofline": {"bound": "alu", "achieved": round(alu_ach, 1), "peak": round(alu_peak, 1),
                        "unit": "Gmodmul/s", "frac": round(alu_ach / alu_peak, 4), "traffic": None,
                        "kernel": "whole exact step (residues, one fused convolution per prime, reconstruction)"},
           "roofline_hbm": {"bound": "hbm", "achieved": round(alg_bytes / (ms * 1e-3) / 1e9, 1), "peak": hbm_peak,
                            "unit": "GB/s", "frac": round(alg_bytes / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                            "peak_src": f"{peak_src} copy bandwidth", "algorithmic_bytes_per_step": alg_bytes},
           "clocks": clk.summary(), "gpu_launches": launches_per_step * steps}
    if not args.quick:
        # end to end: pinned host inputs copied in, exact convolution, result copied out, every step
        fh, gh = f.cpu().pin_memory(), g.cpu().pin_memory()
        hh = torch.empty_like(fh).pin_memory()
        fd, gd = torch.empty_like(f), torch.empty_like(g)
        esteps = max(1, min(args.steps, 20))

        def e2e_step():
            fd.copy_(fh, non_blocking=True)
            gd.copy_(gh, non_blocking=True)
            ntt.conv_exact(plan, fd, gd, out=h, stream=stream)
            hh.copy_(h, non_blocking=True)

        for _ in range(max(args.warmup, 3)):
            e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(esteps):
            e2e_step()
        torch.cuda.synchronize()
        ems = max_over_ranks(world, (time.perf_counter() - t0) * 1000.0 / esteps)
        out["e2e"] = {"value": round(batch * world * 1000.0 / ems, 1), "unit": "conv/s", "ms_per_step": round(ems, 3),
                      "h2d_bytes_per_step": 2 * batch * N * 8, "d2h_bytes_per_step": batch * N * 8,
                      "entry": "conv_exact with torch copies from/to pinned host memory"}
        attach_cpu_baseline(out, "exact6", args, world, rank, full=False)
    return out


def measure_uneven(args, world, rank, local, sub=False):
    """10,000 convolutions of lengths 2^6..2^19 in one batch plan, replayed as
    a CUDA graph; every length class runs its fused kernel."""
    import numpy as np
    import torch

    from paper_1005_1497_gb300 import inputs, ntt

    count = args.batch or WORKLOADS["conv4"][0]
    seed = 1000 + rank
    lens = inputs.log_uniform_lengths(count, 6, 19, seed=seed)
    offs = np.concatenate([[0], np.cumsum(lens)[:-1]])
    total = int(lens.sum())
    f = inputs.uniform_mod_torch(M, total, seed, 0, device="cuda")
    g = inputs.uniform_mod_torch(M, total, seed, 1, device="cuda")
    h = torch.empty_like(f)
    triples = [(f[o:o + n], g[o:o + n], h[o:o + n]) for o, n in zip(offs.tolist(), lens.tolist())]
    if args.tune and not sub:
        schedule = {}
        for k in range(15, 20):                      # split-path classes: autotune form and pairs per wave
            cnt = int((lens == (1 << k)).sum())
            if cnt:
                t = ntt.ntt_autotune(M, 1 << k, cnt)
                schedule[f"2^{k}"] = {"wave": t["wave"], "twist": bool(t["twist"])}
        if args.schedule:
            ntt.ntt_autotune_save(args.schedule)
    else:
        schedule = {}
    bp = ntt.BatchPlan(M, triples)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        bp.exec_graph(stream)
    torch.cuda.synchronize()
    barrier(world)
    steps = max(1, min(args.steps, 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        c0 = ntt.launch_count()
        e0.record(stream)
        for _ in range(steps):
            bp.exec_graph(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = ntt.launch_count() - c0
    ms = max_over_ranks(world, e0.elapsed_time(e1) / steps)
    hbm_peak, sm_max_mhz, peak_src = peaks()
    alg_bytes = 12.0 * total
    L = np.log2(lens).astype(np.int64)
    modmul = float(np.sum(3 * (lens // 2) * L + lens))
    alu_peak = alu_peak_gmodmul(local, sm_max_mhz)
    alu_ach = modmul / (ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": round(count * world * 1000.0 / ms, 1), "unit": "conv/s", "n_gpus": world,
           "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded counter-based)",
           "config": config_of("conv4", args, world), "elements": total, "schedule": schedule,
           "roofline": {"bound": "alu", "achieved": round(alu_ach, 1), "peak": round(alu_peak, 1),
                        "unit": "Gmodmul/s", "frac": round(alu_ach / alu_peak, 4), "traffic": None,
                        "kernel": "all length classes of one step (graph replay); the split classes' rows "
                                  "(k_conv_cr<u32,14,14,·,1>) dominate"},
           "roofline_hbm": {"bound": "hbm", "achieved": round(alg_bytes / (ms * 1e-3) / 1e9, 1), "peak": hbm_peak,
                            "unit": "GB/s", "frac": round(alg_bytes / (ms * 1e-3) / 1e9 / hbm_peak, 4),
                            "peak_src": f"{peak_src} copy bandwidth"},
           "clocks": clk.summary(), "gpu_launches": launches}
    if not args.quick:
        # end to end: each step copies f and g in from pinned host memory (one
        # copy each), replays the batch plan and copies h back
        h_dev = h.clone()
        fh, gh = f.cpu().pin_memory(), g.cpu().pin_memory()
        hh = torch.empty_like(fh).pin_memory()
        esteps = max(1, min(args.steps, 5))
        ew = 3
        for i in range(esteps + ew):
            if i == ew:
                torch.cuda.synchronize()
                barrier(world)
                t0 = time.perf_counter()
            f.copy_(fh, non_blocking=True)
            g.copy_(gh, non_blocking=True)
            bp.exec_graph(stream)
            hh.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        ems = max_over_ranks(world, (time.perf_counter() - t0) * 1000.0 / esteps)
        out["e2e"] = {"value": round(count * world * 1000.0 / ems, 1), "unit": "conv/s", "ms_per_step": round(ems, 3),
                      "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 4 * total,
                      "entry": "ntt_batch_exec_graph between one host-to-device copy of f and of g (pinned) and one "
                               "device-to-host copy of h",
                      "bit_identical_to_device_path": bool(torch.equal(hh, h_dev.cpu()))}
        del fh, gh, hh, h_dev
        attach_cpu_baseline(out, "conv4", args, world, rank, full=not sub)
    bp.close()
    return out


def measure_serve(args, world, rank, local, sub=False):
    """Open-loop Poisson load on the convolution server: requests are
    submitted at their arrival times from pinned host buffers; latency is
    submit -> result back in host memory (p50/p99 from the server)."""
    import numpy as np
    import torch

    from paper_1005_1497_gb300 import inputs, ntt

    m, rate, duration = M64, 20000.0, max(0.5, min(args.steps / 1000.0, 3.0))
    count = int(rate * duration)
    seed = 2000 + rank
    K = 512                                           # distinct request buffers, reused cyclically
    lens = inputs.log_uniform_lengths(K, 8, 18, seed=seed)
    total = int(lens.sum())
    fbuf = inputs.uniform_mod_torch(m, total, seed, 0, device="cuda", dtype=torch.int64).cpu().pin_memory()
    gbuf = inputs.uniform_mod_torch(m, total, seed, 1, device="cuda", dtype=torch.int64).cpu().pin_memory()
    hbuf = torch.empty_like(fbuf).pin_memory()
    offs = [int(v) for v in np.concatenate([[0], np.cumsum(lens)[:-1]])]
    lens = [int(v) for v in lens]
    fp, gp, hp = fbuf.data_ptr(), gbuf.data_ptr(), hbuf.data_ptr()
    gaps = inputs.exponential_gaps(count, rate, seed=seed)
    arrivals = np.cumsum(gaps)
    srv = ntt.Server(m, pool_bytes=2 << 30, streams=4, max_batch=256, max_log2N=18)
    # warm-up: each length once
    for i in range(min(K, 64)):
        st, rid = srv.submit_raw(fp + 8 * offs[i], gp + 8 * offs[i], hp + 8 * offs[i], int(lens[i]))
        srv.wait(rid)
    srv.reset_stats()
    ids = [0] * count
    with ClockSampler(local) as clk:
        c0 = ntt.launch_count()
        t0 = time.perf_counter()
        for i in range(count):
            target = t0 + arrivals[i]
            while time.perf_counter() < target:
                pass
            s = i % K
            if i >= K:
                srv.wait(ids[i - K])                  # buffer reuse: the earlier request is long done
            st, ids[i] = srv.submit_raw(fp + 8 * offs[s], gp + 8 * offs[s], hp + 8 * offs[s], int(lens[s]))
        srv.drain()
        elapsed = time.perf_counter() - t0
        launches = ntt.launch_count() - c0
    stats = srv.stats()
    # capacity: the same requests submitted back to back (closed loop, K in flight)
    srv.reset_stats()
    ccount = min(count, 20000)
    t1 = time.perf_counter()
    cap_ids = [0] * ccount
    for i in range(ccount):
        s = i % K
        if i >= K:
            srv.wait(cap_ids[i - K])
        st, cap_ids[i] = srv.submit_raw(fp + 8 * offs[s], gp + 8 * offs[s], hp + 8 * offs[s], int(lens[s]))
    srv.drain()
    cap_elapsed = time.perf_counter() - t1
    cap = srv.stats()
    srv.close()
    mean_n = float(np.mean(lens))
    out = {"metric": METRIC, "value": round(stats["completed"] / elapsed, 1), "unit": "req/s", "n_gpus": world,
           "steps": count, "warmup": min(K, 64), "ms_per_step": round(elapsed * 1000.0 / count, 4),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
           "data": "synthetic (seeded counter-based; Poisson arrivals)",
           "config": config_of("serve5", args, world),
           "server_config": {"requests": count, "mean_N": round(mean_n, 1), "pool_bytes": 2 << 30, "streams": 4,
                             "max_batch": 256},
           "latency_us": {"p50": round(stats["p50_us"], 1), "p99": round(stats["p99_us"], 1),
                          "mean": round(stats["mean_us"], 1), "max": round(stats["max_us"], 1)},
           "server": {k: stats[k] for k in ("completed", "rejected", "batches", "max_inflight_batches",
                                              "peak_pool_bytes", "direct")},
           "io": "pinned host buffers addressed in place by the kernels (no staging copies)",
           "capacity": {"req_per_s": round(cap["completed"] / cap_elapsed, 1), "requests": ccount,
                        "in_flight": K, "p50_us": round(cap["p50_us"], 1), "p99_us": round(cap["p99_us"], 1),
                        "GBps_host_io": round(24.0 * mean_n * cap["completed"] / cap_elapsed / 1e9, 1)},
           "roofline": {"bound": "latency", "note": "20k req/s of ~48k-word requests offer about 23 GB/s: the "
                                                     "served path is latency-bound, its latency is the figure"},
           "clocks": clk.summary(), "gpu_launches": launches}
    # the serving rate is itself end to end: every request goes from host
    # memory to its result in host memory through ntt_server_submit
    out["e2e"] = {"value": out["value"], "unit": "req/s", "h2d_bytes_per_step": round(16.0 * mean_n, 1),
                  "d2h_bytes_per_step": round(8.0 * mean_n, 1),
                  "entry": "ntt_server_submit / ntt_server_wait on pinned host buffers (a step is one request; "
                           "mean bytes read and written across the host link)"}
    attach_cpu_baseline(out, "serve5", args, world, rank, full=not sub)
    return out


def attach_cpu_baseline(out, name, args, world, rank, full):
    """The oracle on the workload's own pairs, rank 0 at N=1 only, within a
    bounded budget (the full budget for the line's own workload, a quarter
    of it for each attached workload)."""
    if world != 1 or rank != 0:
        return
    out["cpu_baseline"] = cpu_baseline(name, args, args.cpu_seconds if full else args.cpu_seconds / 4, full)


MEASURE = {"conv1": lambda *a, **k: measure_uniform("conv1", *a, **k),
           "conv2": lambda *a, **k: measure_uniform("conv2", *a, **k),
           "conv3": lambda *a, **k: measure_uniform("conv3", *a, **k),
           "conv4": measure_uneven, "serve5": measure_serve, "exact6": measure_exact, "shift7": measure_shift}

# keys of an attached workload's object
SUB_KEYS = ("value", "unit", "ms_per_step", "steps", "config", "roofline", "roofline_hbm", "clocks", "e2e",
            "cpu_baseline", "gpu_launches", "latency_us", "capacity", "server", "schedule", "launch", "noalloc")


def run_ours(args):
    import torch

    from paper_1005_1497_gb300 import ntt
    world, rank, local = dist_setup()
    sched = load_schedule(args, ntt) if not args.tune else {"loaded": None, "tuned": "in this run"}
    out = MEASURE[args.workload](args, world, rank, local)
    out["schedule_file"] = sched
    if args.workload == "conv2" and not args.quick and not args.no_configs and args.log2n is None \
            and args.batch is None:
        configs = {}
        for name in SUB_CONFIGS:
            torch.cuda.empty_cache()
            sub = MEASURE[name](args, world, rank, local, sub=True)
            configs[name] = {k: sub[k] for k in SUB_KEYS if k in sub}
        out["configs"] = configs
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle, as it stands, timed on the host cores on bounded samples of
    the same workload (rank 0 only): its radix-2 convolution on whole pairs,
    threads over pairs (exact integer workloads: direct Eq. 1 on sampled
    outputs)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pairs, unit = reference_pairs(args.workload, args)
    per_step = max(1.0, min(5.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_rate_mixed(pairs, per_step / 4, kind="fast")
    rates, total, thr = [], 0, 1
    for _ in range(args.steps):
        r, thr, done, _ = oracle_rate_mixed(pairs, per_step, kind="fast")
        rates.append(r)
        total += done
    value = statistics.median(rates)
    integer = pairs[0][3] == "int"
    what = ("exact integer Eq. 1 in 128-bit integers on sampled outputs" if integer else
            "the oracle's radix-2 convolution (or_fast_conv) on whole pairs, threads over pairs")
    sample = (f"{what}: {total} {'outputs' if integer else 'pair convolutions'} over {len(pairs)} pairs of the "
              f"workload, {per_step:.1f} s per step; rate = threads x pairs / sum of each pair's time")
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": unit, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000.0 * per_step, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64 (oracle, __int128 products)",
           "data": "synthetic (seeded counter-based)",
           "config": config_of(args.workload, args, args.gpus),
           "cpu_baseline": {"value": round(value, 4), "unit": unit, "cores": thr, "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
