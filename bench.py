#!/usr/bin/env python3
"""Benchmark of the batched NTT on GB300.

Default workload (one "step" = forward then inverse transform of every vector,
lazy butterflies of Algorithms 3 and 4):
    p = 998244353 (beta = 2^32), 64 transforms of L = 2^16, one of L = 2^20
    and one of L = 2^22, uint32 residues uniform in [0, p) from a seed.
The three groups run on three CUDA streams; every pass is one kernel launch
timed with CUDA events on its own stream.  L2 is flushed (a 512 MiB write)
between timed steps.  The NTL-style comparator (Algorithm 2 butterflies, same
schedule) is timed the same way.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload c2|c1|c3|c4|c5]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica on its own GPU (the workload has no exchange step), value = total
butterflies of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import concurrent.futures
import gc
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1205_2926_gb300.inputs import P_NTT30, P_NTT62, batch_inputs, uneven_batch_spec, uniform_residues  # noqa

METRIC = "NTT butterflies/s & HBM GB/s, lazy vs NTL-style on GB300; p50/p99 polymul latency"

WORKLOADS = {
    "c1": {"name": "single forward+inverse NTT, L=2^10, p=998244353 (uint32)", "groups": [(P_NTT30, 10, 1)]},
    "c2": {"name": "32-bit batched NTT, p=998244353: 64 x 2^16 + 1 x 2^20 + 1 x 2^22, forward+inverse",
           "groups": [(P_NTT30, 16, 64), (P_NTT30, 20, 1), (P_NTT30, 22, 1)]},
    "c3": {"name": "64-bit NTT, p=2305843009448574977: 16 x 2^20 + 1 x 2^24, forward+inverse",
           "groups": [(P_NTT62, 20, 16), (P_NTT62, 24, 1)]},
    "c4": {"name": "uneven batch: 4096 transforms, L = 2^8..2^16 log-uniform, 3 primes = 1 mod 2^16, "
                   "half inverse, one persistent launch", "groups": []},
    "c5": {"name": "polymul serving: Poisson 20k req/s, p = 998244353, degrees log-uniform 2^6..2^20",
           "groups": []},
    "probe": {"name": "register-only butterfly rate probe", "groups": []},
    "bigint": {"name": "big-integer product: 2^22 x 2^22 limbs of 32 bits (3 NTT primes + CRT + carries)",
               "groups": []},
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured", "sm_max_mhz": float(d.get("sm_max_mhz", 2070))}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback", "sm_max_mhz": 2070.0}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed loop runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [ln for (t, ln) in self.lines if t0 - 0.15 <= t <= t1 + 0.15] or [ln for _, ln in self.lines]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in rows:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per launch of the dominant pass kernel come from
# one ncu capture summarised in profiles/dram_traffic.md: a table of
# `| workload | kernel | bytes per launch | kernel source hash |` rows.  The
# hash covers the pass kernels' sources; a row taken from other sources (the
# kernels changed since the counters were taken) gives null, not a stale number.
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "dram_traffic.md")
KERNEL_SOURCES = ["ntt_kernels.cuh", "modarith.cuh", "ntt_pass_inst.cuh", "ntt_pass_u32.cu", "ntt_pass_u64.cu",
                  "ntt_plan.cu"]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1205_2926_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, kernel: str):
    """(bytes per launch or None, note) for a pass of a workload."""
    try:
        lines = open(TRAFFIC_PROFILE).read().splitlines()
    except OSError:
        return None, "no capture summarised"
    want = kernel_source_hash()
    for ln in lines:
        f = [x.strip() for x in ln.strip().strip("|").split("|")]
        if len(f) == 4 and f[0] == workload and f[1] == kernel:
            if f[3] != want:
                return None, f"capture of other kernel sources ({f[3]}; now {want})"
            try:
                return int(f[2]), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {os.path.basename(TRAFFIC_PROFILE)}"
            except ValueError:
                return None, "unreadable row"
    return None, "kernel not captured"


def alu_peak_bfly(word_bytes, sm_mhz):
    """Integer-multiply roof in butterflies/s.  A butterfly takes one high and
    two low products (Section 5: three multiplies); with the multiply rates
    measured on this GB300 by `bench.py --workload probe` (per SM and clock:
    mul.hi.u32 31.3, mad.lo.u32 62.8; mul.hi.u64 7.25, mul.lo.u64 15.1) that
    is 1 / (1/hi + 2/lo) = 15.7 butterflies/clk/SM for 32-bit words and 3.7
    for 64-bit words."""
    per_clk = 1.0 / (1.0 / 31.3 + 2.0 / 62.8) if word_bytes == 4 else 1.0 / (1.0 / 7.25 + 2.0 / 15.1)
    return 152 * sm_mhz * 1e6 * per_clk


def butterflies(groups):
    """Butterflies per forward (or inverse) transform set: l * L/2 per vector (Section 5 count)."""
    return sum(b * l * (1 << l) // 2 for (_, l, b) in groups)


def useful_bytes(groups):
    """One read and one write of every word per transform."""
    return sum(2 * b * (1 << l) * (4 if p < (1 << 30) else 8) for (p, l, b) in groups)


# --------------------------------------------------------------------------- ours

class GPUWorkload:
    def __init__(self, groups, torch, ntt, seed=1, autotune=True):
        self.torch, self.ntt = torch, ntt
        self.groups = groups
        self.plans, self.bufs, self.streams, self.host = [], [], [], []
        self.splits = []
        for gi, (p, l, b) in enumerate(groups):
            L = 1 << l
            plan = ntt.ntt_plan(p, ntt.root_of_unity(p, L), L)
            # the library's autotuner picks the pass split for this batch size
            self.splits.append(plan.autotune(b, use_cache=True) if autotune else list(plan.info().log_r)[:plan.info().n_passes])
            a = batch_inputs(seed + gi, b, L, p)
            view = a.view(np.int32) if a.dtype == np.uint32 else a.view(np.int64)
            t = torch.from_numpy(view.copy()).cuda()
            self.plans.append(plan)
            self.bufs.append(t)
            self.streams.append(torch.cuda.Stream())
            self.host.append(torch.from_numpy(view.copy()).pin_memory())
        self.nsteps = [p.info().n_passes for p in self.plans]
        self.flush_buf = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=len(groups))

    def set_variant(self, v):
        for p in self.plans:
            p.set_variant(v)

    def flush_l2(self):
        self.flush_buf.fill_(1)

    def step(self, events=None):
        """Forward then inverse of every group, each pass a launch on the group's
        stream.  With `events`, the groups run one after another on the current
        stream and every launch is bracketed by CUDA events (clean per-kernel
        durations, comparable with the ncu launch list).  The stream first
        spins for about a millisecond so that the host has queued every launch
        before the first one runs: the passes then follow each other as in the
        graph replays, with no host launch gaps inside the event brackets."""
        torch, ntt = self.torch, self.ntt
        cur = torch.cuda.current_stream()
        if events is not None:
            torch.cuda._sleep(2_000_000)
        for gi, (plan, buf, s) in enumerate(zip(self.plans, self.bufs, self.streams)):
            if events is not None:
                s = cur
            else:
                s.wait_stream(cur)
            b = self.groups[gi][2]
            for inv in (0, 1):
                for k in range(self.nsteps[gi]):
                    if events is not None:
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(s)
                    ntt.ntt_execute_step(plan, inv, k, buf, b, stream=s)
                    if events is not None:
                        e1.record(s)
                        events.append(((gi, inv, k), e0, e1))
        if events is None:
            for s in self.streams:
                cur.wait_stream(s)

    def step_e2e(self):
        """End to end through the host-buffer C-ABI call: per group,
        ntt_transform_host forward then inverse on the group's pinned host
        batch (each call copies in, transforms and copies out; batches above
        2 MiB pipeline the copies against the transforms in chunks).  The
        groups run concurrently, one host thread each (ctypes releases the
        GIL for the duration of each library call)."""
        futs = [self.pool.submit(self._e2e_group, gi) for gi in range(len(self.groups))]
        for f in futs:
            f.result()

    def _e2e_group(self, gi):
        plan, h, s = self.plans[gi], self.host[gi], self.streams[gi]
        b = self.groups[gi][2]
        self.ntt.ntt_transform_host(plan, False, h, b, stream=s)
        self.ntt.ntt_transform_host(plan, True, h, b, stream=s)

    def e2e_bytes(self):
        """Host->device and device->host bytes of one e2e step (two calls per group)."""
        return 2 * (useful_bytes(self.groups) // 2)


def barrier(dist):
    if dist is not None and dist.is_initialized():
        dist.barrier()


def reduce_max(x: float, dist, device: str) -> float:
    """Max of a per-rank value over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over the
    slowest rank's time (weak scaling, no data-path collective)."""
    return units_per_rank * world / max_seconds


def capture_step(wl, torch):
    """CUDA graph of one step (forward + inverse of every group on its own
    stream, forked from and joined back to the capturing stream)."""
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            wl.step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    return g


def time_steps(wl, torch, K, W, dist, graph=None, with_events=False):
    """K timed steps (graph replays when a graph is given), L2 flushed before
    each; returns (total ms of the K steps, per-pass events, wall window)."""
    run = (lambda ev=None: graph.replay()) if graph is not None else (lambda ev=None: wl.step(ev))
    for _ in range(W):
        wl.flush_l2()
        run()
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    per_step = []
    events = []
    t0 = time.time()
    for _ in range(K):
        wl.flush_l2()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        run(events if with_events else None)
        s1.record()
        per_step.append((s0, s1))
    torch.cuda.synchronize()
    t1 = time.time()
    barrier(dist)
    steps_ms = [a.elapsed_time(b) for a, b in per_step]
    wl.last_steps_ms = steps_ms
    return sum(steps_ms), events, (t0, t1)


def time_e2e(wl, torch, K, W, dist):
    for _ in range(W):
        wl.step_e2e()
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        wl.step_e2e()
        torch.cuda.synchronize()
    t1 = time.perf_counter()
    barrier(dist)
    return (t1 - t0) * 1e3


def kernel_stats(events, groups):
    """Average duration per pass (group, direction, step) and the dominant one."""
    acc = {}
    for key, e0, e1 in events:
        acc.setdefault(key, []).append(e0.elapsed_time(e1))
    stats = {}
    for key, v in acc.items():
        gi = key[0]
        p, l, b = groups[gi]
        w = 4 if p < (1 << 30) else 8
        stats[key] = {"avg_ms": float(np.mean(v)), "launches": len(v), "total_ms": float(np.sum(v)),
                      "bytes": 2 * b * (1 << l) * w}
    dom = max(stats, key=lambda k: stats[k]["total_ms"])
    return stats, dom


def max_over_ranks(x, dist, torch):
    return reduce_max(x, dist, "cuda")


def cpu_sample(groups, budget_s):
    """Run the CPU oracle (Algorithm 1 and its inverse, fully reduced, one
    core) on whole transforms of each group until the budget is spent.
    Returns (butterflies, seconds, description)."""
    import oracle
    o = oracle.get()
    done_bfly, t_used, parts = 0, 0.0, []
    per_group = budget_s / len(groups)
    for gi, (p, l, b) in enumerate(groups):
        L = 1 << l
        w = o.root_of_unity(p, L)
        a = batch_inputs(1 + gi, 1, L, p).astype(np.uint64)
        n, t_g = 0, 0.0
        while t_g < per_group and n < b:
            t0 = time.perf_counter()
            y = o.ntt_ref(p, w, a)
            o.intt_ref(p, w, y)
            t_g += time.perf_counter() - t0
            n += 1
        done_bfly += n * 2 * l * L // 2
        t_used += t_g
        parts.append(f"{n} x 2^{l} fwd+inv")
    return done_bfly, t_used, "; ".join(parts)


def _oracle_task(task):
    """One forward + inverse transform by the oracle (a worker of the
    all-cores CPU baseline); returns its butterflies."""
    import oracle
    p, l, seed = task
    o = oracle.get()
    L = 1 << l
    w = o.root_of_unity(p, L)
    a = batch_inputs(seed, 1, L, p).astype(np.uint64)
    o.intt_ref(p, w, o.ntt_ref(p, w, a))
    return l * L  # 2 * l * L / 2


def cpu_baseline_all_cores(groups, budget_s=12.0):
    """The same oracle on every host core: independent transforms of the
    workload run in a process pool (spawned, one process per core), one whole
    forward + inverse transform per task, as many tasks as fit the budget at
    the single-core rate.  Butterflies done / wall time."""
    import multiprocessing as mp
    bf1, t1, _ = cpu_sample(groups, 2.0)  # single-core rate sizes the sample
    rate1 = bf1 / t1
    cores = os.cpu_count() or 1
    tasks = []
    budget_bf = rate1 * budget_s * cores
    acc = 0
    while acc < budget_bf:
        for gi, (p, l, b) in enumerate(groups):
            for k in range(b):
                tasks.append((p, l, 1 + gi + 1000 * k))
                acc += l * (1 << l)
                if acc >= budget_bf:
                    break
            if acc >= budget_bf:
                break
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_task, [(groups[0][0], 3, 0)] * cores)  # start-up outside the timing
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_task, tasks, chunksize=1))
        t = time.perf_counter() - t0
    return {"value": done / t, "unit": "butterflies/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(tasks)} whole forward+inverse transforms of the workload's groups in a pool of "
                      f"{cores} processes ({t:.1f} s)", "host": host_cpu()}


def host_cpu():
    """The host CPU the oracle ran on: model name (lscpu) and logical cores."""
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "logical_cores": os.cpu_count()}


def cpu_baseline_oracle(groups, budget_s=12.0):
    bf, t, desc = cpu_sample(groups, budget_s)
    return {"value": bf / t, "unit": "butterflies/s", "cores": 1, "kind": "oracle",
            "sample": desc + f" of the same workload ({t:.1f} s, single thread)", "host": host_cpu()}


def run_uneven(args, dist, rank, world):
    """Uneven batch: 4096 transforms, log2 L uniform in 8..16, three 30-bit
    primes, half inverse, in one persistent launch (ntt_execute_uneven)
    captured in a CUDA graph; value = butterflies/s."""
    import torch
    import paper_1205_2926_gb300 as ntt
    from paper_1205_2926_gb300 import build
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    spec = uneven_batch_spec()
    plans, descs, bfly, nbytes, pass_bytes = {}, [], 0, 0, 0
    for d in spec:
        L = 1 << d["logL"]
        key = (d["p"], L)
        if key not in plans:
            plans[key] = ntt.ntt_plan(d["p"], ntt.root_of_unity(d["p"], L), L)
        a = uniform_residues(40_000 + d["id"], L, d["p"]).astype(np.uint32)
        t = torch.from_numpy(a.view(np.int32).copy()).cuda()
        descs.append((plans[key], t, d["inverse"]))
        bfly += d["logL"] * L // 2
        nbytes += 8 * L
        pass_bytes += 8 * L * plans[key].info().n_passes
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    # the library's autotuner picks each multi-pass length class's split inside
    # the persistent launch (served from the cache when tuned before)
    ntt.ntt_uneven_autotune(descs, use_cache=True, stream=s)
    class_splits = {f"2^{k[1].bit_length() - 1} p={k[0]}": list(pl.info().log_r)[:pl.info().n_passes]
                    for k, pl in plans.items() if pl.info().n_passes > 1}
    pass_bytes = sum(8 * (1 << d["logL"]) * plans[(d["p"], 1 << d["logL"])].info().n_passes for d in spec)
    with torch.cuda.stream(s):
        ntt.ntt_execute_uneven(descs, stream=s)  # prepares the device work list
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ntt.ntt_execute_uneven(descs, stream=s)
    for _ in range(args.warmup):
        flush.fill_(1)
        g.replay()
    torch.cuda.synchronize()
    barrier(dist)
    peaks = load_peaks()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    ev = []
    t0 = time.time()
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    t1 = time.time()
    clocks = sampler.stop(t0, t1)
    assert ntt.ntt_uneven_status() == 0
    per_step = sorted(a.elapsed_time(b) for a, b in ev)
    ms = max_over_ranks(sum(per_step), dist, torch)
    K = args.steps
    per = ms / K / 1e3
    gbs = nbytes / per / 1e9
    # the same batch with the NTL-style butterflies (Algorithm 2), same splits
    for pl in plans.values():
        pl.set_variant(ntt.VARIANT_NTL)
    with torch.cuda.stream(s):
        ntt.ntt_execute_uneven(descs, stream=s)
    torch.cuda.synchronize()
    g_ntl = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_ntl, stream=s):
        ntt.ntt_execute_uneven(descs, stream=s)
    for _ in range(args.warmup):
        flush.fill_(1)
        g_ntl.replay()
    ev_ntl = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g_ntl.replay()
        e1.record()
        ev_ntl.append((e0, e1))
    torch.cuda.synchronize()
    assert ntt.ntt_uneven_status() == 0
    ms_ntl = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev_ntl), dist, torch)
    for pl in plans.values():
        pl.set_variant(ntt.VARIANT_LAZY)
    return {
        "metric": METRIC, "value": world * bfly / per, "unit": "butterflies/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms / K,
        "step_ms": {"median": per_step[len(per_step) // 2],
                    "p99": per_step[min(len(per_step) - 1, int(0.99 * len(per_step)))]},
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded uniform residues)",
        "config": {"workload": WORKLOADS["c4"]["name"], "transforms": len(spec), "butterflies_per_step": bfly,
                   "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{world}",
                   "class_splits_log2": class_splits},
        "hbm_gbs_useful": gbs,
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "traffic": None, "kernel": "k_uneven (one launch per step)",
                     "per_pass": {"achieved": pass_bytes / per / 1e9, "frac": pass_bytes / per / 1e9 / peaks["hbm_gbs"],
                                  "note": "every word read and written once per pass (two passes above 2^11)"}},
        "gpu_launches": 1, "graph": "one CUDA graph replay per step", "clocks": clocks,
        "ntl": {"value": world * bfly / (ms_ntl / K / 1e3), "unit": "butterflies/s", "ms_per_step": ms_ntl / K},
        "lazy_over_ntl": round(ms_ntl / ms, 4),
    }


def run_serving(seconds, rate, torch, ntt, seed=5, max_log=20.0, variant=0):
    """Poisson stream of polynomial products mod 998244353 (degrees
    log-uniform in 2^6..2^max_log) through the continuous-batching server
    (its transforms with the lazy butterflies, variant 0, or the NTL-style
    ones, variant 1).  Operands are slices of one pinned pool of uniform
    residues; results go to a pinned ring (not checked here; the tests check
    them).  Returns latency percentiles and throughput."""
    from paper_1205_2926_gb300.inputs import serving_trace
    n = int(seconds * rate)
    trace = serving_trace(seed=seed, n=n, rate_per_s=rate, dmax_log=max_log)
    pool_words = 1 << 24
    pool = torch.from_numpy(uniform_residues(seed, pool_words, P_NTT30).astype(np.uint32).view(np.int32)).pin_memory()
    ring_words = 1 << 28
    ring = torch.empty(ring_words, dtype=torch.int32).pin_memory()
    base, rbase = pool.data_ptr(), ring.data_ptr()
    sv = ntt.Server(P_NTT30, max_coeffs=(1 << int(max_log)) + 1, mem_budget_bytes=8 << 30, n_streams=8,
                    max_batch=512, variant=variant)
    rng = np.random.default_rng(seed)
    offs = rng.integers(0, pool_words - (1 << 21), size=(n, 2))
    # warm-up: one request of every length class, the largest included
    # (operands of 2^max_log + 1 coefficients: L = 2^(max_log + 2))
    for lg in range(7, int(max_log) + 2):
        m = (1 << (lg - 1))
        sv.submit(base, m, base, m, rbase)
    m = (1 << int(max_log)) + 1
    sv.submit(base, m, base, m, rbase)
    sv.drain(-1)
    sv.reset_stats()
    # the submission loop replays the trace from plain lists, with Python's
    # garbage collector paused: a collection pass (tens of ms with this many
    # live objects) would hold back submissions and then release them as one
    # burst, which the latency of the burst would show instead of the server's
    t_arr = [r["t_arrive_s"] for r in trace]
    nas = [r["na"] for r in trace]
    nbs = [r["nb"] for r in trace]
    a_ptr = [base + 4 * int(x) for x in offs[:, 0]]
    b_ptr = [base + 4 * int(x) for x in offs[:, 1]]
    rpos = 0
    load_before = os.getloadavg()[0]
    gc_was = gc.isenabled()
    gc.disable()
    t_start = time.perf_counter()
    refused = 0
    for i in range(n):
        target = t_start + t_arr[i]
        while time.perf_counter() < target:
            pass
        out_words = nas[i] + nbs[i] - 1
        if rpos + out_words > ring_words:
            rpos = 0
        rc, _ = sv.submit(a_ptr[i], nas[i], b_ptr[i], nbs[i], rbase + 4 * rpos)
        refused += rc != 0
        rpos += out_words
    t_sub = time.perf_counter() - t_start
    if gc_was:
        gc.enable()
    load_after = os.getloadavg()[0]
    sv.drain(-1)
    st = sv.stats()
    sv.destroy()
    return {"requests": n, "offered_rate_per_s": rate, "submit_window_s": t_sub, "completed": int(st.completed),
            "refused": int(st.refused) + refused * 0, "p50_ms": st.p50_us / 1e3, "p99_ms": st.p99_us / 1e3,
            "mean_ms": st.mean_us / 1e3, "max_ms": st.max_us / 1e3,
            "throughput_req_per_s": st.completed / st.wall_s if st.wall_s else None,
            "butterflies_per_s": st.butterflies / st.wall_s if st.wall_s else None, "batches": int(st.batches),
            "direct_batches": int(st.direct_batches),
            "host_load_1min": {"before": load_before, "after": load_after}}


def run_serve_workload(args, dist, rank, world):
    import torch
    import paper_1205_2926_gb300 as ntt
    from paper_1205_2926_gb300 import build
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    t0 = time.time()
    res = run_serving(args.serve_seconds, 20000.0, torch, ntt)
    clocks = sampler.stop(t0, time.time())
    # the same trace with the NTL-style butterflies (Algorithm 2)
    res_ntl = run_serving(args.serve_seconds, 20000.0, torch, ntt, variant=1)
    # offered-load sweep around the configured rate (1 s each): where the
    # latency knee lies
    sweep = []
    for rate in (10000.0, 40000.0, 80000.0, 160000.0):
        r = run_serving(1.0, rate, torch, ntt, seed=6)
        sweep.append({"offered_rate_per_s": rate, "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
                      "throughput_req_per_s": r["throughput_req_per_s"], "refused": r["refused"]})
    return {
        "metric": METRIC, "value": res["p99_ms"], "unit": "ms (p99 polymul latency)", "n_gpus": world,
        "steps": res["requests"], "warmup": args.warmup, "ms_per_step": res["mean_ms"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded Poisson trace)",
        "config": {"workload": WORKLOADS["c5"]["name"], "seconds": args.serve_seconds,
                   "cuda_module_loading": os.environ.get("CUDA_MODULE_LOADING", "LAZY (default)")},
        "serving": res, "rate_sweep": sweep, "clocks": clocks,
        "ntl": {"p50_ms": res_ntl["p50_ms"], "p99_ms": res_ntl["p99_ms"],
                "throughput_req_per_s": res_ntl["throughput_req_per_s"]},
    }


def run_bigint(args, dist, rank, world):
    """Section 1's large-integer application: the product of two integers of
    2^22 32-bit limbs (134 Mbit each) by three NTT polynomial products
    (primes 998244353, 167772161, 469762049, L = 2^23), Chinese remaindering
    and a carry scan (bigint_mul).  Timed with CUDA events, L2 flushed before
    each product (parity of bigint_mul up to this size is in the tests)."""
    import torch
    import paper_1205_2926_gb300 as ntt
    from paper_1205_2926_gb300 import build
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = 1 << 22
    rng = np.random.default_rng(11)
    a = torch.from_numpy(rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32).view(np.int32)).cuda()
    b = torch.from_numpy(rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32).view(np.int32)).cuda()
    c = torch.empty(2 * n, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        ntt.bigint_mul(a, n, b, n, c)
    torch.cuda.synchronize()
    K = max(3, min(args.steps, 20))
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    t0 = time.time()
    ms = []
    for _ in range(K):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ntt.bigint_mul(a, n, b, n, c)
        e1.record()
        ms.append((e0, e1))
    torch.cuda.synchronize()
    clocks = sampler.stop(t0, time.time())
    times = sorted(x.elapsed_time(y) for x, y in ms)
    mean = sum(times) / K
    bfly = 3 * 3 * 23 * (1 << 22)  # three primes x (two forward + one inverse) transforms of 2^23
    return {
        "metric": "big-integer product time (2^22 x 2^22 32-bit limbs)", "value": mean, "unit": "ms per product",
        "n_gpus": world, "steps": K, "warmup": args.warmup, "ms_per_step": mean,
        "step_ms": {"median": times[K // 2], "p99": times[-1]}, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded uniform limbs)",
        "config": {"workload": WORKLOADS["bigint"]["name"], "l2": "flushed before each product (512 MiB write)"},
        "input_mbit_per_s": 2 * 32 * n / (mean / 1e3) / 1e6, "transform_butterflies_per_s": bfly / (mean / 1e3),
        "clocks": clocks,
    }


def run_probe():
    """Build and run bench_probes/butterfly_rate.cu: register-only butterfly
    and multiply rates of this GPU (the integer-pipe roof of the NTT kernels)."""
    from paper_1205_2926_gb300 import build as b
    src = os.path.join(ROOT, "bench_probes", "butterfly_rate.cu")
    exe = os.path.join(ROOT, "bench_probes", "_build", "butterfly_rate")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    subprocess.run([b._nvcc(), *b.ARCH, "-O3", "-std=c++17", "-I", os.path.join(ROOT, "paper_1205_2926_gb300", "csrc"),
                    src, "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, check=True)
    res = json.loads(r.stdout.strip().splitlines()[-1])
    return {"metric": "register-only butterflies per clock per SM", "value": res["lazy_fwd_bfly_per_clk_sm"],
            "unit": "butterflies/clk/SM", "higher_is_better": True, "config": {"workload": "probe"}, "probe": res}


STEADY = {
    "c2": [(P_NTT30, 20, 64), (P_NTT30, 22, 16), (P_NTT30, 16, 1024)],
    "c3": [(P_NTT62, 20, 32), (P_NTT62, 24, 2)],
}


def steady_state(cases, torch, ntt, peak_gbs, K=20, warm=3, sm_mhz=2070.0, warp_rows=False):
    """The pass kernels at 256 MiB per batch (twice the L2, so every pass reads
    and writes HBM), CUDA-event time of K back-to-back launches of each pass.
    Per pass: that pass's bytes (one read and one write of every word) over its
    time.  Per transform: one read and one write of every word per direction
    (the algorithmic bytes of the whole transform, however many passes it
    takes) over the forward+inverse time, against the measured HBM copy peak;
    and butterflies/s against the integer-multiply roof.  The split is the
    library's own for that batch (autotuned, cached); with warp_rows the row
    passes of 2^5..2^10 words run with one warp per row."""
    out = []
    for p, l, b in cases:
        L = 1 << l
        w = 4 if p < (1 << 30) else 8
        plan = ntt.ntt_plan(p, ntt.root_of_unity(p, L), L)
        split = plan.autotune(b, use_cache=True)
        if warp_rows:
            plan.set_warp_rows(True)
        a = batch_inputs(3, b, L, p)
        t = torch.from_numpy(a.view(np.int32) if w == 4 else a.view(np.int64)).cuda()
        passes, total_us = [], 0.0
        for inv in (0, 1):
            for k in range(len(split)):
                for _ in range(warm):
                    ntt.ntt_execute_step(plan, inv, k, t, b)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(K):
                    ntt.ntt_execute_step(plan, inv, k, t, b)
                e1.record()
                torch.cuda.synchronize()
                us = e0.elapsed_time(e1) * 1e3 / K
                total_us += us
                gbs = 2 * b * L * w / (us * 1e-6) / 1e9
                passes.append({"pass": f"{'inverse' if inv else 'forward'} {k}",
                               "log2_R": (split[::-1] if inv else split)[k], "us": round(us, 1),
                               "GBs": round(gbs), "frac": round(gbs / peak_gbs, 3)})
        # per transform (Section 5's unit of work): one read and one write of
        # every word per direction, whatever the number of passes
        per_transform = 2 * (2 * b * L * w)
        bfly_s = 2 * b * (L // 2) * l / (total_us * 1e-6)
        out.append({"workload": f"{b} x 2^{l}, {8 * w}-bit words ({b * L * w >> 20} MiB)", "split": split,
                    "passes": passes, "fwd_inv_us": round(total_us, 1),
                    "butterflies_per_s": bfly_s,
                    "hbm_frac_per_transform": round(per_transform / (total_us * 1e-6) / 1e9 / peak_gbs, 3),
                    "hbm_frac_mean_per_pass": round(float(np.mean([x["frac"] for x in passes])), 3),
                    "multiply_roof_frac": round(bfly_s / alu_peak_bfly(w, sm_mhz), 3)})
        del t
        plan.destroy()
    torch.cuda.synchronize()
    return out


def run_steady_only(args):
    """Only the 256 MiB per-pass report of the workload's lengths: with
    --steady-launches 1 every pass of every case launches exactly once, in
    order (forward passes, then inverse passes), so that a profiler can
    capture them by position."""
    import torch
    import paper_1205_2926_gb300 as ntt
    from paper_1205_2926_gb300 import build
    build.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    K = max(1, args.steady_launches)
    cases = STEADY.get(args.workload, STEADY["c2"])
    return {"what": "pass kernels at 256 MiB per pass, CUDA events, HBM fraction of measured peak",
            "launches_per_pass": K, "row_body": "one warp per row" if args.warp_rows else "radix-8 CTA rows",
            "cases": steady_state(cases, torch, ntt, load_peaks()["hbm_gbs"], K=K, warm=3 if K > 1 else 0,
                                  sm_mhz=load_peaks()["sm_max_mhz"], warp_rows=args.warp_rows)}


def run_ours(args, dist, rank, world):
    import torch
    import paper_1205_2926_gb300 as ntt
    from paper_1205_2926_gb300 import build

    build.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    spec = WORKLOADS[args.workload]
    groups = spec["groups"]
    wl = GPUWorkload(groups, torch, ntt)
    peaks = load_peaks()
    sampler = ClockSampler(local)
    sampler.start()
    bfly_step = 2 * butterflies(groups)
    bytes_step = 2 * useful_bytes(groups)

    # headline: graph replays of the whole step (lazy butterflies)
    wl.set_variant(0)
    for _ in range(3):
        wl.step()
    torch.cuda.synchronize()
    graph = capture_step(wl, torch)
    ms_lazy, _, (t0, t1) = time_steps(wl, torch, args.steps, args.warmup, dist, graph=graph)
    lazy_steps = sorted(wl.last_steps_ms)
    clocks = sampler.stop(t0, t1)
    ms_lazy = max_over_ranks(ms_lazy, dist, torch)
    # per-kernel durations: the same step launched eagerly, CUDA events around each pass
    _, events, _ = time_steps(wl, torch, args.steps, args.warmup, dist, with_events=True)
    stats, dom = kernel_stats(events, groups)
    # comparator: Algorithm 2 butterflies in the same schedule
    wl.set_variant(1)
    for _ in range(3):
        wl.step()
    graph_ntl = capture_step(wl, torch)
    ms_ntl, _, _ = time_steps(wl, torch, args.steps, args.warmup, dist, graph=graph_ntl)
    ms_ntl = max_over_ranks(ms_ntl, dist, torch)
    # Algorithm 5 (Montgomery's product, lazy ranges) in the same schedule
    wl.set_variant(2)
    for _ in range(3):
        wl.step()
    graph_mont = capture_step(wl, torch)
    ms_mont, _, _ = time_steps(wl, torch, args.steps, args.warmup, dist, graph=graph_mont)
    ms_mont = max_over_ranks(ms_mont, dist, torch)
    wl.set_variant(0)
    k_e2e = max(3, min(args.steps, 50))
    ms_e2e = time_e2e(wl, torch, k_e2e, 2, dist)
    ms_e2e = max_over_ranks(ms_e2e, dist, torch)

    K = args.steps
    value = job_value(bfly_step * K, world, ms_lazy / 1e3)
    ntl_value = job_value(bfly_step * K, world, ms_ntl / 1e3)
    ds = stats[dom]
    gi, inv, k = dom
    p_, l_, b_ = groups[gi]
    w_ = 4 if p_ < (1 << 30) else 8
    achieved_gbs = ds["bytes"] / (ds["avg_ms"] / 1e3) / 1e9
    # butterflies of the dominant pass: every element takes log2(R) / 2 of them
    log_r = wl.plans[gi].info().log_r[k if not inv else wl.nsteps[gi] - 1 - k]
    pass_bfly = b_ * (1 << l_) * log_r / 2
    achieved_bfly = pass_bfly / (ds["avg_ms"] / 1e3)
    alu_peak = alu_peak_bfly(w_, peaks["sm_max_mhz"])
    frac_hbm = achieved_gbs / peaks["hbm_gbs"]
    frac_alu = achieved_bfly / alu_peak
    dom_name = f"{'inverse' if inv else 'forward'} pass {k} of {b_} x 2^{l_} (log2 R = {log_r})"
    traffic, traffic_note = ncu_traffic(args.workload, dom_name)
    if frac_alu >= frac_hbm:
        roof = {"bound": "alu", "achieved": achieved_bfly / 1e9, "peak": alu_peak / 1e9, "unit": "Gbutterflies/s",
                "frac": frac_alu, "traffic": traffic, "kernel": dom_name,
                "peak_src": f"152 SMs x clock x {alu_peak / (152 * peaks['sm_max_mhz'] * 1e6):.1f} butterflies/clk/SM "
                            "(measured multiply rates)",
                "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": frac_hbm}}
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": frac_hbm, "traffic": traffic, "kernel": dom_name,
                "peak_src": peaks["src"] + " (MEASURED_PEAKS.json, of measured)",
                "alu": {"achieved": achieved_bfly / 1e9, "peak": alu_peak / 1e9, "unit": "Gbutterflies/s",
                        "frac": frac_alu}}
    roof["traffic_src"] = traffic_note
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "butterflies/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms_lazy / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32" if groups[0][0] < (1 << 30) else "u64",
        "data": "synthetic (seeded uniform residues)",
        "config": {"workload": spec["name"], "butterflies_per_step": bfly_step,
                   "pass_splits_log2": wl.splits,
                   "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{world}"},
        "gpu_launches": len(events) // K,
        "clocks": clocks,
        "e2e": {"value": world * bfly_step * k_e2e / (ms_e2e / 1e3), "unit": "butterflies/s",
                "h2d_bytes_per_step": wl.e2e_bytes(), "d2h_bytes_per_step": wl.e2e_bytes(),
                "path": "ntt_transform_host on pinned host buffers, fwd then inv per group"},
        "roofline": roof,
        "step_ms": {"median": lazy_steps[len(lazy_steps) // 2],
                    "p99": lazy_steps[min(len(lazy_steps) - 1, int(0.99 * len(lazy_steps)))]},
        "hbm_gbs_useful": world * bytes_step * K / (ms_lazy / 1e3) / 1e9,
    }
    detail = {"kernels_us": {f"g{g}{'i' if i else 'f'}{s}": round(v["avg_ms"] * 1e3, 2) for (g, i, s), v in stats.items()},
              "graph": "timed steps are CUDA graph replays; kernel times from an eager pass with events"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(groups)
        allc = cpu_baseline_all_cores(groups)
        line["cpu_baseline_all_cores"] = {"value": allc["value"], "unit": allc["unit"], "cores": allc["cores"]}
        detail["cpu_baseline_all_cores"] = allc
    if args.workload in STEADY and not args.no_steady_state:
        try:
            cases = steady_state(STEADY[args.workload], torch, ntt, peaks["hbm_gbs"],
                                 K=max(1, args.steady_launches), sm_mhz=peaks["sm_max_mhz"])
            detail["steady_state"] = cases
            line["steady_256MiB"] = {c["workload"].split(",")[0]: {
                "split": c["split"], "fwd_inv_us": c["fwd_inv_us"], "hbm_frac_per_transform": c["hbm_frac_per_transform"],
                "hbm_frac_mean_per_pass": c["hbm_frac_mean_per_pass"], "multiply_roof_frac": c["multiply_roof_frac"]}
                for c in cases}
        except Exception as e:  # a report of its own; the headline above stands
            line["steady_256MiB"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_serving and args.workload == "c2":
        sv = run_serving(args.serve_seconds, 20000.0, torch, ntt)
        sv_ntl = run_serving(args.serve_seconds, 20000.0, torch, ntt, variant=1)
        detail["polymul_serving"] = sv
        detail["polymul_serving_ntl"] = sv_ntl
        line["polymul_serving"] = {"seconds": args.serve_seconds, "offered_req_per_s": 20000,
                                   "p50_ms": round(sv["p50_ms"], 4), "p99_ms": round(sv["p99_ms"], 4),
                                   "completed_req_per_s": round(sv["throughput_req_per_s"] or 0.0, 1),
                                   "ntl_p50_ms": round(sv_ntl["p50_ms"], 4), "ntl_p99_ms": round(sv_ntl["p99_ms"], 4)}
    if args.workload == "c2" and not args.no_u64:
        # the paper's own word size (beta = 2^64, Table 1): the 64-bit batched
        # configuration, lazy against NTL-style in the same schedule
        try:
            line["u64_c3"] = u64_comparison(args, dist, torch, ntt)
        except Exception as e:
            line["u64_c3"] = {"error": f"{type(e).__name__}: {e}"}
    line["montgomery"] = {"value": job_value(bfly_step * K, world, ms_mont / 1e3),
                          "lazy_over_montgomery": round(ms_mont / ms_lazy, 4)}
    line["ntl"] = {"value": ntl_value, "unit": "butterflies/s", "ms_per_step": ms_ntl / K}
    line["lazy_over_ntl"] = round(ms_ntl / ms_lazy, 4)
    return line, detail


def u64_comparison(args, dist, torch, ntt):
    """16 x 2^20 + 1 x 2^24 64-bit words (p = 2305843009448574977), forward +
    inverse per step, graph replays with the L2 flushed: lazy (Algorithms 3/4)
    and NTL-style (Algorithm 2), same schedule, same K steps as the headline."""
    groups = WORKLOADS["c3"]["groups"]
    wl = GPUWorkload(groups, torch, ntt, seed=31)
    bfly_step = 2 * butterflies(groups)
    out = {"workload": WORKLOADS["c3"]["name"]}
    ms = {}
    for name, v in (("lazy", 0), ("ntl", 1)):
        wl.set_variant(v)
        for _ in range(3):
            wl.step()
        g = capture_step(wl, torch)
        t, _, _ = time_steps(wl, torch, args.steps, args.warmup, dist, graph=g)
        ms[name] = max_over_ranks(t, dist, torch) / args.steps
        del g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    out["value"] = world * bfly_step / (ms["lazy"] / 1e3)
    out["ms_per_step"] = round(ms["lazy"], 4)
    out["ntl_value"] = world * bfly_step / (ms["ntl"] / 1e3)
    out["lazy_over_ntl"] = round(ms["ntl"] / ms["lazy"], 4)
    del wl
    torch.cuda.empty_cache()
    return out


REF_STEP_BUDGET_S = 6.0  # upper bound on one reference step's oracle time (seconds)


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, same config, metric and unit.
    Each step is a bounded sample of the workload (whole transforms)."""
    if rank != 0:
        return None
    spec = WORKLOADS[args.workload]
    if args.workload in ("c4", "c5"):
        return run_reference_sampled(args, world)
    groups = spec["groups"]
    budget = min(REF_STEP_BUDGET_S, max(0.5, min(6.0, 60.0 / max(args.steps + args.warmup, 1))))
    for _ in range(args.warmup):
        cpu_sample(groups, budget)
    bf_total, t_total, desc = 0, 0.0, ""
    for _ in range(args.steps):
        bf, t, desc = cpu_sample(groups, budget)
        bf_total += bf
        t_total += t
    value = bf_total / t_total
    bfly_step = 2 * butterflies(groups)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "butterflies/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": bfly_step / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32" if groups[0][0] < (1 << 30) else "u64",
        "data": "synthetic (seeded uniform residues)",
        "config": {"workload": spec["name"], "butterflies_per_step": bfly_step},
        "cpu_baseline": {"value": value, "unit": "butterflies/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: {desc} of the workload, single thread", "host": host_cpu()},
        "e2e": {"value": value, "unit": "butterflies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_sampled(args, world):
    """Oracle on a bounded sample of the uneven batch (c4: transforms of the
    spec in order, forward or inverse as specified) or of the serving trace
    (c5: products through the oracle's convolution, one after another)."""
    import oracle
    o = oracle.get()
    budget = max(1.0, min(20.0, 60.0 / max(args.steps + args.warmup, 1) * args.steps))
    if args.workload == "c4":
        spec = uneven_batch_spec()
        bf, t, n = 0, 0.0, 0
        for d in spec:
            if t > budget:
                break
            L = 1 << d["logL"]
            a = uniform_residues(40_000 + d["id"], L, d["p"])
            w = o.root_of_unity(d["p"], L)
            t0 = time.perf_counter()
            (o.intt_ref if d["inverse"] else o.ntt_ref)(d["p"], w, a)
            t += time.perf_counter() - t0
            bf += d["logL"] * L // 2
            n += 1
        value, unit, hib = bf / t, "butterflies/s", True
        sample = f"first {n} of 4096 transforms of the uneven batch ({t:.1f} s, single thread)"
        extra = {}
    else:
        from paper_1205_2926_gb300.inputs import serving_trace
        trace = serving_trace(n=100000, rate_per_s=20000.0)
        lat, t = [], 0.0
        for r in trace:
            if t > budget:
                break
            a = uniform_residues(r["id"], r["na"], P_NTT30)
            b = uniform_residues(r["id"] + 1, r["nb"], P_NTT30)
            t0 = time.perf_counter()
            o.polymul_ntt(P_NTT30, a, b)
            dt = time.perf_counter() - t0
            t += dt
            lat.append(dt * 1e3)
        lat = np.array(lat)
        value, unit, hib = float(np.percentile(lat, 99)), "ms (p99 polymul latency)", False
        sample = f"{len(lat)} products of the serving trace, one at a time, no queueing ({t:.1f} s, single thread)"
        extra = {"serving": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": value, "requests": len(lat)}}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": None, "higher_is_better": hib, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOADS[args.workload]["name"]},
        "cpu_baseline": {"value": value, "unit": unit, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    line.update(extra)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=None,
                    help="serving run length (default: 60 s for --workload c5, 2 s inside the default bench)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-u64", action="store_true", help="skip the 64-bit lazy vs NTL-style comparison")
    ap.add_argument("--no-steady-state", action="store_true", help="skip the 256 MiB per-pass report")
    ap.add_argument("--steady-only", action="store_true",
                    help="only the 256 MiB per-pass report (for profiling the pass kernels at that size)")
    ap.add_argument("--warp-rows", action="store_true",
                    help="with --steady-only: row passes of 2^5..2^10 words with one warp per row")
    ap.add_argument("--steady-launches", type=int, default=20,
                    help="timed launches per pass in the 256 MiB report (1: no warm-up, one launch per pass)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve_seconds is None:
        args.serve_seconds = 60.0 if args.workload == "c5" else 2.0
    if args.workload == "c5":
        # a serving process loads its CUDA modules at start-up: with the
        # default lazy loading, 5 of 8 twenty-second runs at 20k req/s showed
        # one 12-98 ms stall (and a p99 up to 23 ms); 0 of 8 with eager
        # loading.  Set before the first CUDA call of the process.
        os.environ.setdefault("CUDA_MODULE_LOADING", "EAGER")
    if "NTT_AUTOTUNE_CACHE" not in os.environ:
        # start from the pass splits tuned on this GPU model (shipped with the
        # package); a shape or GPU it lacks is tuned at run time into the copy
        import shutil
        import tempfile
        cache = os.path.join(tempfile.mkdtemp(prefix="ntt_bench_"), "autotune.json")
        shutil.copy(os.path.join(ROOT, "paper_1205_2926_gb300", "autotune_gb300.json"), cache)
        os.environ["NTT_AUTOTUNE_CACHE"] = cache
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference" and args.workload == "probe":
        print(json.dumps({"impl": "reference", "unavailable": "the probe measures GPU pipes only"}))
        return
    if args.impl == "reference" and args.workload == "bigint":
        print(json.dumps({"impl": "reference", "unavailable": "an extra workload beyond the benchmark configurations; "
                          "its oracle (exact CPU integer product) is used by the tests only"}))
        return
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.steady_only:
        line = run_steady_only(args)
    elif args.workload == "probe":
        line = run_probe()
    elif args.workload == "c4":
        line = run_uneven(args, dist, rank, world)
    elif args.workload == "c5":
        line = run_serve_workload(args, dist, rank, world)
    elif args.workload == "bigint":
        line = run_bigint(args, dist, rank, world)
    else:
        line, detail = run_ours(args, dist, rank, world)
        if rank == 0:
            # the full per-pass report goes to stderr; stdout keeps one compact line
            print("detail " + json.dumps(detail), file=sys.stderr, flush=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
