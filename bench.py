#!/usr/bin/env python3
"""Benchmark: sorted keys/s of the bitonic network, melded vs divergent kernels.

One step = one whole sort (every pass of the network) of one synthetic array
already resident in HBM.  Default workload: 2^26 float32 keys (N(0,1) with 1 %
exact duplicates and signed zeros, ordered by the IEEE-754 totalOrder bit
map), the paper's 2^26-element bitonic input.  `--workload kv24` runs the
key-value sort of 2^24 uniform uint32 keys with a uint32 payload (payload =
index).

Prints ONE JSON line on rank 0.  Under torchrun (N > 1) every rank sorts its
own replica (the network of one array does not shard without an exchange
step): weak scaling, value = arrays sorted by all ranks / max time.

--impl reference times the CPU oracle (single-threaded plain C of the
same network) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sorted keys/s, melded vs divergent bitonic kernel; warp exec efficiency"
L2_FLUSH_BYTES = 256 << 20  # larger than the 126 MiB L2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["darm", "reference"], default="darm")
    ap.add_argument("--workload",
                    choices=["kv24", "kv24skew", "f32", "cfg1", "oem4096", "oem26", "pcm28",
                             "sb", "seg", "serve"],
                    default="f32")
    ap.add_argument("--serve-requests", type=int, default=3000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def workload(name):
    """(description, keys, vals, dtype label) for a workload name."""
    import synth
    if name == "kv24":
        k, v = synth.cfg2_kv(skew=False)
        return ("bitonic key-value sort, 2^24 uint32 keys uniform, uint32 payload = index", k, v)
    if name == "kv24skew":
        k, v = synth.cfg2_kv(skew=True)
        return ("bitonic key-value sort, 2^24 uint32 keys = rand mod 16, uint32 payload = index",
                k, v)
    if name == "cfg1":
        return ("single-block bitonic sort, 4096 uint32 keys uniform (the paper's Fig. 1 kernel), "
                "one thread block", synth.cfg1_keys(), None)
    k = synth.cfg3_f32()
    return ("bitonic sort, 2^26 float32 keys N(0,1) with 1% duplicates and signed zeros", k, None)


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"darm_bench_clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args, backend="nccl"):
    """Rank layout from torchrun's environment.  Ranks are independent
    replicas (the whole-array network does not shard without an exchange
    step); the process group only carries the barrier and the max of the
    timings."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, world, rank):
    """CPU oracle on a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    import oracle
    desc, keys, vals = workload(args.workload)
    n_full = keys.size
    # bounded sample: a power-of-two prefix of the same array, sized so that
    # W + K sorts stay within a few minutes on one core
    budget_s = 150.0
    per_ce_ns = 4.5
    steps = args.steps + args.warmup
    m = int(np.log2(n_full))
    while m > 10 and oracle.compare_exchanges(1 << m) * per_ce_ns * 1e-9 * steps > budget_s:
        m -= 1
    n = 1 << m
    ks = keys[:n].copy()
    vs = None if vals is None else vals[:n].copy()
    for _ in range(args.warmup):
        oracle.bitonic_sort(ks, vs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.bitonic_sort(ks, vs)
    dt = (time.perf_counter() - t0) / args.steps
    value = n / dt
    sample = f"first 2^{m} elements of the {n_full}-element array, one oracle sort per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if vals is None and keys.dtype == np.float32 else
        "u32", "data": "synthetic",
        "config": {"workload": desc, "n": n_full},
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "sample": sample, "host": host_cpu()},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_sources_sha256():
    """Hash of the pass kernels' sources and of the planner that shapes their
    launches; a recorded DRAM traffic figure is used only while these are
    unchanged since it was captured (host-side code such as the C ABI entry
    points, batching and serving does not enter)."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2107_05681_gb300", "csrc")
    names = ["*.cuh", "kernel_table.h", "plan.h", "plan.cu", "kernels_*.cu", "tile_*.cu",
             "tma_*.cu", "window2*.cu"]
    files = sorted({f for pat in names for f in glob.glob(os.path.join(csrc, pat))})
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(workload_name, pass_kind):
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_sources_sha256") != kernel_sources_sha256():
        return None
    return rec.get(workload_name, {}).get(pass_kind)


def measured_hbm_peak():
    """HBM copy bandwidth (GB/s) measured on this machine's GPUs, else the
    earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def cpu_baseline(keys, vals):
    """Oracle keys/s on a bounded sample (about 10-20 s of one core)."""
    import numpy as np

    import oracle
    n_full = keys.size
    m = int(np.log2(n_full))
    while m > 12 and oracle.compare_exchanges(1 << m) * 4.5e-9 > 15.0:
        m -= 1
    n = 1 << m
    ks = keys[:n].copy()
    vs = None if vals is None else vals[:n].copy()
    reps, dt = 0, 0.0
    while dt < 1.0:  # small arrays: repeat the sort for at least a second
        t0 = time.perf_counter()
        oracle.bitonic_sort(ks, vs)
        dt += time.perf_counter() - t0
        reps += 1
    what = "one" if reps == 1 else f"{reps}"
    # the textbook routine beside it: numpy's single-threaded sort of the same
    # keys (keys only)
    t0 = time.perf_counter()
    lib_reps = 0
    while time.perf_counter() - t0 < 0.5:
        np.sort(keys[:n], kind="quicksort")
        lib_reps += 1
    lib_dt = time.perf_counter() - t0
    return {"value": reps * n / dt, "unit": "keys/s", "cores": 1, "kind": "oracle",
            "sample": f"{what} single-threaded oracle sort(s) of the first 2^{m} elements "
                      f"({dt:.1f} s)",
            "library_sort_keys_per_s": lib_reps * n / lib_dt,
            "library_sort": "numpy.sort (introsort, one thread), keys only",
            "host": host_cpu()}


def host_cpu():
    """Core count and CPU model of this host."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or
            platform.machine()}


def run_oddeven(args, world, rank, local):
    """Batcher's odd-even merge sort network (the base of the paper's PCM
    benchmark), melded vs divergent, L2 flushed between sorts: one thread
    block on 4096 uniform uint32 keys (oem4096), or 2^26 uniform uint32 keys
    sorted bucket by bucket, 4096 keys per thread block (oem26, the paper's
    way of running its benchmarks on a 2^26-element input)."""
    import numpy as np
    import torch

    import oracle
    import paper_2107_05681_gb300 as darm
    import synth
    bucket = 4096
    if args.workload == "oem26":
        keys = synth.uniform_u32(0xDA2C0006, 1 << 26)
        what = ("Batcher odd-even merge sort network, 2^26 uint32 keys uniform, sorted in "
                "buckets of 4096 keys, one thread block per bucket")
    else:
        keys = synth.cfg1_keys()
        what = "Batcher odd-even merge sort network, 4096 uint32 keys uniform, one thread block"
    n = keys.size
    src = torch.from_numpy(keys).cuda()
    work = torch.empty_like(src)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    def run_sort(t, variant="melded"):
        darm.oddeven_sort_buckets(t, bucket=bucket, variant=variant)

    work.copy_(src)
    run_sort(work)
    torch.cuda.synchronize()
    got = work.cpu().numpy().reshape(-1, bucket)
    assert np.all(got[:, 1:] >= got[:, :-1]), "a bucket is not sorted"
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    out, launches = {}, 0
    for variant in ("melded", "divergent"):
        for _ in range(args.warmup):
            work.copy_(src)
            run_sort(work, variant)
        torch.cuda.synchronize()
        barrier(world)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        l0 = darm.launch_count()
        for a, b in evs:
            work.copy_(src)
            flush.fill_(1.0)
            a.record(stream)
            run_sort(work, variant)
            b.record(stream)
        torch.cuda.synchronize()
        launches += darm.launch_count() - l0
        out[variant] = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world)
    clk = clocks.stop()
    # end to end through the binding: pinned host -> device, sort, back
    hk = torch.empty(n, dtype=torch.uint32, pin_memory=True)
    tot = 0.0
    for _ in range(args.steps):
        hk.copy_(torch.from_numpy(keys))
        t0 = time.perf_counter()
        work.copy_(hk, non_blocking=True)
        run_sort(work)
        hk.copy_(work, non_blocking=True)
        torch.cuda.synchronize()
        tot += time.perf_counter() - t0
    tot = max_over_ranks(tot, world)
    if rank == 0:
        ms = out["melded"]
        if n > bucket:
            # every key is read and written once: 8 bytes per key per sort
            ach = 8.0 * n * args.steps / (ms * 1e-3) / 1e9
            peak = measured_hbm_peak()
            roof = {"bound": "shared memory + barriers (78 layers per bucket)",
                    "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": None, "note": "HBM traffic of one sort: one read and one write "
                    "of each key; the time is the buckets' in-block layers"}
        else:
            roof = {"bound": "latency", "note": "one CTA on one SM: 78 layers, two barriers "
                    "each; HBM and ALU peaks do not bound it"}
        t0, reps = time.perf_counter(), 0
        while time.perf_counter() - t0 < 1.0:  # one bucket per oracle call
            oracle.oddeven_sort(keys[(reps % (n // bucket)) * bucket:][:bucket])
            reps += 1
        cdt = time.perf_counter() - t0
        line = {
            "metric": "sorted keys/s, melded vs divergent odd-even merge sort network; warp exec "
                      "efficiency",
            "value": world * n * args.steps / (ms * 1e-3), "unit": "keys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": what, "n": n, "bucket": bucket, "variant": "melded",
                       "l2": "flushed between steps (256 MiB write outside the timed events)"},
            "divergent": {"value": world * n * args.steps / (out["divergent"] * 1e-3),
                          "ms_per_step": out["divergent"] / args.steps},
            "melded_over_divergent": out["divergent"] / ms,
            "roofline": roof,
            "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": world * n * args.steps / tot, "unit": "keys/s",
                    "h2d_bytes_per_step": n * 4, "d2h_bytes_per_step": n * 4},
            "cpu_baseline": {"value": reps * bucket / cdt, "unit": "keys/s", "cores": 1,
                             "kind": "oracle", "host": host_cpu(),
                             "sample": f"{reps} single-threaded oracle runs of the network, "
                                       f"one {bucket}-key bucket each ({cdt:.1f} s)"},
        }
        print(json.dumps(line), flush=True)


def pcm_layer_bytes(n, bucket):
    """Algorithmic HBM bytes of PCM's merge-split layers over n uint32 keys:
    every comparator reads and writes its two buckets once (8 bytes per key
    moved); layer (s, t) of B buckets has B/2 comparators when t == s, else
    (B / 2^(s+1)) (2^s - 2^t).  Returns (total bytes, layer launches)."""
    nb = n // bucket
    total, launches = 0, 0
    s = 0
    while (1 << s) < nb:
        for t in range(s, -1, -1):
            ncmp = nb // 2 if t == s else (nb >> (s + 1)) * ((1 << s) - (1 << t))
            total += ncmp * 2 * bucket * 8
            launches += 1
        s += 1
    return total, launches


def run_pcm(args, world, rank, local):
    """PCM (Section VI-A): 2^28 uniform uint32 keys, buckets of 4096 sorted by
    the odd-even merge sort network, then odd-even merged bucket by bucket
    with merge-splits; melded vs divergent merge loop, L2 flushed between
    sorts."""
    import numpy as np
    import torch

    import oracle
    import paper_2107_05681_gb300 as darm
    import synth
    bucket = 4096
    keys = synth.uniform_u32(0xDA2C0008, 1 << 28)
    n = keys.size
    src = torch.from_numpy(keys).cuda()
    work = torch.empty_like(src)
    scratch = torch.empty_like(src)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def run_sort(t, variant="melded"):
        darm.pcm_sort(t, bucket=bucket, scratch_keys=scratch, variant=variant)

    work.copy_(src)
    run_sort(work)
    torch.cuda.synchronize()
    got = work.cpu().numpy()
    assert np.all(got[1:] >= got[:-1]), "PCM result not sorted"
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    out, launches = {}, 0
    for variant in ("melded", "divergent"):
        for _ in range(args.warmup):
            work.copy_(src)
            run_sort(work, variant)
        torch.cuda.synchronize()
        barrier(world)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        l0 = darm.launch_count()
        for a, b in evs:
            work.copy_(src)
            flush.fill_(1.0)
            a.record(stream)
            run_sort(work, variant)
            b.record(stream)
        torch.cuda.synchronize()
        launches += darm.launch_count() - l0
        out[variant] = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world)
    # the bucket sorts alone, to split the time between the two kernels
    bevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(args.steps)]
    for a, b in bevs:
        work.copy_(src)
        flush.fill_(1.0)
        a.record(stream)
        darm.oddeven_sort_buckets(work, bucket=bucket)
        b.record(stream)
    torch.cuda.synchronize()
    bucket_ms = sum(a.elapsed_time(b) for a, b in bevs) / args.steps
    clk = clocks.stop()
    # end to end: pinned host -> device, sort, back
    hk = torch.empty(n, dtype=torch.uint32, pin_memory=True)
    hk.copy_(src.cpu())
    tot = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        work.copy_(hk, non_blocking=True)
        run_sort(work)
        hk.copy_(work, non_blocking=True)
        torch.cuda.synchronize()
        tot += time.perf_counter() - t0
    tot = max_over_ranks(tot, world)
    if rank == 0:
        ms = out["melded"] / args.steps
        layer_bytes, nlayers = pcm_layer_bytes(n, bucket)
        layers_ms = ms - bucket_ms
        ach = layer_bytes / (layers_ms * 1e-3) / 1e9
        peak = measured_hbm_peak()
        # CPU baseline: the oracle on a bounded prefix (2^20 keys, 256 buckets)
        m_cpu = 20
        t0, reps = time.perf_counter(), 0
        while time.perf_counter() - t0 < 2.0:
            oracle.pcm_sort(keys[: 1 << m_cpu], bucket=bucket)
            reps += 1
        cdt = time.perf_counter() - t0
        line = {
            "metric": "sorted keys/s, PCM (odd-even merge of sorted buckets), melded vs "
                      "divergent merge loop",
            "value": world * n / (ms * 1e-3), "unit": "keys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "PCM, 2^28 uint32 keys uniform, buckets of 4096 keys "
                                   "(65,536 buckets), the paper's PCM input size",
                       "n": n, "bucket": bucket, "variant": "melded",
                       "l2": "flushed between steps (256 MiB write outside the timed events)"},
            "divergent": {"value": world * n * args.steps / (out["divergent"] * 1e-3),
                          "ms_per_step": out["divergent"] / args.steps},
            "melded_over_divergent": out["divergent"] / out["melded"],
            "roofline": {"bound": "hbm", "kernel": "merge-split layers", "achieved": ach,
                         "peak": peak, "unit": "GB/s", "frac": ach / peak, "traffic": None,
                         "algorithmic_bytes": layer_bytes / nlayers, "layers": nlayers,
                         "layers_ms": layers_ms, "bucket_sort_ms": bucket_ms,
                         "note": "achieved = algorithmic bytes of all merge-split layers / their "
                                 "time (the sort's time minus the bucket sorts' time)"},
            "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": world * n * args.steps / tot, "unit": "keys/s",
                    "h2d_bytes_per_step": n * 4, "d2h_bytes_per_step": n * 4},
            "cpu_baseline": {"value": reps * (1 << m_cpu) / cdt, "unit": "keys/s", "cores": 1,
                             "kind": "oracle", "host": host_cpu(),
                             "sample": f"{reps} single-threaded oracle PCM sorts of the first "
                                       f"2^{m_cpu} keys ({cdt:.1f} s)"},
        }
        print(json.dumps(line), flush=True)


def run_synthetic(args, world, rank, local):
    """The synthetic divergent kernels SB1, SB4, SB1-R, SB4-R (Section VI-A),
    melded vs divergent: 1216 blocks of 256 threads (eight per SM), 64 outer
    iterations of 4 divergent inner steps, 32 compute rounds per path."""
    import math

    import numpy as np
    import torch

    import oracle
    import paper_2107_05681_gb300 as darm
    import synth
    nblocks, iters, rounds = 152 * 8, 64, 32
    src = torch.from_numpy(synth.uniform_u32(0xDA2C0007, 1024 * nblocks)).cuda()
    work = torch.empty_like(src)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    # correctness guard: the first 8 blocks against the oracle
    sample = src[: 8 * 1024].cpu().numpy()
    for pat in darm.SB_PATTERNS:
        work.copy_(src)
        darm.sb_run(pat, work, iters, rounds)
        torch.cuda.synchronize()
        assert np.array_equal(work[: 8 * 1024].cpu().numpy(),
                              oracle.sb_run(pat, sample, iters, rounds)), pat
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    res, launches = {}, 0
    for pat in darm.SB_PATTERNS:
        res[pat] = {}
        for variant in ("melded", "divergent"):
            for _ in range(args.warmup):
                work.copy_(src)
                darm.sb_run(pat, work, iters, rounds, variant=variant)
            torch.cuda.synchronize()
            barrier(world)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            l0 = darm.launch_count()
            for a, b in evs:
                work.copy_(src)
                flush.fill_(1.0)
                a.record(stream)
                darm.sb_run(pat, work, iters, rounds, variant=variant)
                b.record(stream)
            torch.cuda.synchronize()
            launches += darm.launch_count() - l0
            res[pat][variant] = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs),
                                               world) / args.steps
    clk = clocks.stop()
    speedups = {p: r["divergent"] / r["melded"] for p, r in res.items()}
    geo = math.exp(sum(math.log(v) for v in speedups.values()) / len(speedups))
    # end to end: copy in, all four kernels (melded), copy back
    hk = torch.empty(src.numel(), dtype=torch.uint32, pin_memory=True)
    hk.copy_(src.cpu())
    tot = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        work.copy_(hk, non_blocking=True)
        for pat in darm.SB_PATTERNS:
            darm.sb_run(pat, work, iters, rounds)
        hk.copy_(work, non_blocking=True)
        torch.cuda.synchronize()
        tot += time.perf_counter() - t0
    tot = max_over_ranks(tot, world)
    if rank == 0:
        t0, reps = time.perf_counter(), 0
        while time.perf_counter() - t0 < 1.0:
            oracle.sb_run("SB1", sample[:1024], iters, rounds)
            reps += 1
        cdt = time.perf_counter() - t0
        per_block_steps = 256 * iters * 4  # thread inner steps per block
        line = {
            "metric": "synthetic divergent kernels: melded over divergent speedup (geomean of "
                      "SB1, SB4, SB1-R, SB4-R); warp exec efficiency",
            "value": geo, "unit": "x", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(r["melded"] for r in res.values()),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "synthetic divergent kernels SB1, SB4, SB1-R, SB4-R, "
                                   f"{nblocks} blocks x 256 threads, {iters} outer iterations, "
                                   f"4 divergent inner steps, {rounds} rounds per path",
                       "l2": "flushed between steps (256 MiB write outside the timed events)"},
            "per_kernel_ms": res, "speedup": speedups,
            "paper_context": "DARM on an AMD Vega 20: 1.36x geomean over SB1-SB4(-R)",
            "roofline": {"bound": "alu", "note": "compute rounds in registers; shared memory "
                         "traffic 2 loads + 1 store per path step"},
            "clocks": clk, "gpu_launches": launches,
            "e2e": {"value": world * nblocks * per_block_steps * 4 * args.steps / tot,
                    "unit": "thread inner steps/s (all four kernels, copies included)",
                    "h2d_bytes_per_step": src.numel() * 4, "d2h_bytes_per_step": src.numel() * 4},
            "cpu_baseline": {"value": reps * per_block_steps / cdt,
                             "unit": "thread inner steps/s (SB1)", "cores": 1, "kind": "oracle",
                             "host": host_cpu(),
                             "sample": f"{reps} oracle runs of SB1 on one block ({cdt:.1f} s)"},
        }
        print(json.dumps(line), flush=True)


def run_segmented(args, world, rank, local):
    """Batched segmented sort: 10,000 uint32 arrays, log-uniform real lengths
    32..65536 padded to powers of two, one graph replay per step."""
    import numpy as np
    import torch

    import paper_2107_05681_gb300 as darm
    import synth
    segs = synth.cfg4_segments()
    real = int(segs.lengths.astype(np.int64).sum())
    padded = int(segs.offsets[-1])
    src_k = torch.from_numpy(segs.keys).cuda()
    src_v = torch.from_numpy(segs.vals).cuda()
    k, v = torch.empty_like(src_k), torch.empty_like(src_v)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    out = {}
    launches = 0
    tuned = None
    for variant in ("melded", "divergent", "auto"):
        if variant == "auto":
            # the batch autotuner (outside the timed region) picks tile size,
            # window depth and the form per pass kind for this layout
            import tempfile
            with tempfile.TemporaryDirectory() as td:
                db = os.path.join(td, "seg.db")
                k.copy_(src_k)
                v.copy_(src_v)
                darm.autotune_segmented(k, v, segs.offsets, segs.lengths, db)
                f = open(db).read().split()
            names = ["key_kind", "payload", "log2n", "tile_log2", "e_tile_log2", "e_window_log2",
                     "window_threads_log2", "windows_per_pass", "bulk_copy_buffers",
                     "form_tile", "form_window", "form_merge"]
            tuned = dict(zip(names, (int(x) for x in f[:12])))
            for kf in ("form_tile", "form_window", "form_merge"):
                tuned[kf] = "melded" if tuned[kf] == 1 else "divergent"
            tuned["tuner_ms"] = float(f[12])
            for i, key in ((13, "shuffle"), (14, "e_merge_log2"), (15, "merge_tile_log2")):
                if len(f) > i:
                    tuned[key] = int(f[i])
        for _ in range(args.warmup):
            k.copy_(src_k)
            v.copy_(src_v)
            darm.segmented_sort(k, v, segs.offsets, segs.lengths, variant=variant)
        torch.cuda.synchronize()
        barrier(world)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        l0 = darm.launch_count()
        for a, b in evs:
            k.copy_(src_k)
            v.copy_(src_v)
            flush.fill_(1.0)
            a.record(stream)
            darm.segmented_sort(k, v, segs.offsets, segs.lengths, variant=variant)
            b.record(stream)
        torch.cuda.synchronize()
        launches += darm.launch_count() - l0
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world)
        out[variant] = ms
    if rank == 0:
        ms = out["melded"]
        line = {
            "metric": "batched segmented sort: real keys/s (melded vs divergent)",
            "value": world * real * args.steps / (ms * 1e-3), "unit": "keys/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "10,000 uint32 key-value segments, real lengths log-uniform "
                                   "32..65536, sentinel-padded to powers of two",
                       "real_keys": real, "padded_keys": padded,
                       "l2": "flushed between steps"},
            "padded_keys_per_s": world * padded * args.steps / (ms * 1e-3),
            "divergent": {"value": world * real * args.steps / (out["divergent"] * 1e-3),
                          "ms_per_step": out["divergent"] / args.steps},
            "autotuned": {"value": world * real * args.steps / (out["auto"] * 1e-3),
                          "ms_per_step": out["auto"] / args.steps, "tuning": tuned},
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)


def run_serving(args, world, rank, local):
    """Poisson arrivals of uint64 key-value sort requests, sizes 2^U(8,20),
    mixed directions, 4 GB budget: saturated throughput, then p50/p99 latency
    at 50/80/95 % of it, for both kernel forms."""
    import threading

    import numpy as np
    import torch

    import paper_2107_05681_gb300 as darm
    import synth
    count = args.serve_requests
    reqs = synth.cfg5_requests(count=count, materialize=False)
    bank = torch.from_numpy(synth.uniform_u64(synth.SEED_CFG5, 1 << 21)).cuda()
    idx = torch.from_numpy(np.arange(1 << 20, dtype=np.uint32)).cuda()
    offs = synth.below(synth.substream(synth.SEED_CFG5, 9), count, 1 << 20)

    def make(r, i):
        k = bank[int(offs[i]):int(offs[i]) + r.n].clone()
        v = idx[:r.n].clone()
        return k, v

    def run(variant, rate):
        darm.serve_start(budget_bytes=4 << 30, max_inflight=256, variant=variant,
                         num_streams=2)
        bufs = [make(r, i) for i, r in enumerate(reqs)]
        torch.cuda.synchronize()
        ids = [None] * count
        t0 = time.perf_counter()
        if rate is None:
            for i, ((k, v), r) in enumerate(zip(bufs, reqs)):
                ids[i] = darm.serve_submit(k, v, descending=r.desc)
        else:
            gaps = -np.log(synth.uniform01(synth.substream(synth.SEED_CFG5, 11), count)) / rate
            t = 0.0
            for i, ((k, v), r) in enumerate(zip(bufs, reqs)):
                t += gaps[i]
                dt = t0 + t - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                ids[i] = darm.serve_submit(k, v, descending=r.desc)
        for rid in ids:
            darm.serve_wait(rid, 600000)
        wall = time.perf_counter() - t0
        p50, p99, kps, done = darm.serve_stats()
        darm.serve_stop()
        keys = sum(r.n for r in reqs)
        return {"p50_ms": p50, "p99_ms": p99, "keys_per_s": keys / wall,
                "offered_req_per_s": rate, "completed": done}

    res = {}
    for variant in ("melded", "divergent"):
        sat = run(variant, None)
        req_rate = count / (sum(r.n for r in reqs) / sat["keys_per_s"])
        loads = {}
        for frac in (0.5, 0.8, 0.95):
            loads[str(frac)] = run(variant, frac * req_rate)
        res[variant] = {"saturated": sat, "loads": loads}
    if rank == 0:
        line = {
            "metric": "serving: keys/s and p50/p99 latency, melded vs divergent",
            "value": res["melded"]["saturated"]["keys_per_s"], "unit": "keys/s",
            "n_gpus": world, "steps": count, "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"{count} uint64 key-value sort requests, sizes 2^U(8,20), "
                                   "direction Bernoulli(0.5), 4 GB budget, Poisson arrivals",
                       "max_inflight": 256, "streams": 2},
            "melded": res["melded"], "divergent": res["divergent"],
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload in ("seg", "serve", "oem4096", "oem26", "pcm28", "sb"):
        import torch

        import paper_2107_05681_gb300 as darm
        torch.cuda.set_device(local)
        darm.init(local)
        runner = {"seg": run_segmented, "serve": run_serving, "oem4096": run_oddeven,
                  "oem26": run_oddeven, "pcm28": run_pcm, "sb": run_synthetic}
        runner[args.workload](args, world, rank, local)
        return
    import numpy as np
    import torch

    import paper_2107_05681_gb300 as darm

    torch.cuda.set_device(local)
    darm.init(local)
    desc, keys_np, vals_np = workload(args.workload)
    n = keys_np.size
    has_vals = vals_np is not None
    dtype_code = darm.F32 if keys_np.dtype == np.float32 else darm.U32
    elem_bytes = keys_np.itemsize + (4 if has_vals else 0)

    src_k = torch.from_numpy(keys_np).cuda()
    src_v = torch.from_numpy(vals_np).cuda() if has_vals else None
    work_k = torch.empty_like(src_k)
    work_v = torch.empty_like(src_v) if has_vals else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def reset():
        work_k.copy_(src_k)
        if has_vals:
            work_v.copy_(src_v)
        flush.fill_(1.0)  # evicts the array from L2 between steps

    def timed_steps(variant, steps, warmup):
        for _ in range(warmup):
            reset()
            darm.sort(work_k, work_v, variant=variant)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        l0 = darm.launch_count()
        for a, b in evs:
            reset()
            a.record(stream)
            darm.sort(work_k, work_v, variant=variant)
            b.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        launches = darm.launch_count() - l0
        ms = sum(a.elapsed_time(b) for a, b in evs)
        return ms, launches

    # correctness guard on the timed configuration (cheap properties; the
    # element-by-element parity against the oracle lives in the tests)
    reset()
    darm.sort(work_k, work_v, variant="melded")
    torch.cuda.synchronize()
    got = work_k.cpu().numpy()
    if keys_np.dtype == np.float32:
        gw = got.view(np.uint32)
        mapped = np.where((gw >> np.uint32(31)) != 0, ~gw, gw | np.uint32(0x80000000))
        assert np.all(mapped[1:] >= mapped[:-1]), "result not sorted"
    else:
        assert np.all(got[1:] >= got[:-1]), "result not sorted"

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)  # let the sampler start before the timed region
    ms_meld, launches_meld = timed_steps("melded", args.steps, args.warmup)
    ms_div, launches_div = timed_steps("divergent", args.steps, args.warmup)
    clk = clocks.stop()
    ms_meld = max_over_ranks(ms_meld, world)
    ms_div = max_over_ranks(ms_div, world)
    value = world * n * args.steps / (ms_meld * 1e-3)
    value_div = world * n * args.steps / (ms_div * 1e-3)

    # per-launch timing for the roofline of the dominant pass kind
    passes, launches_per_sort, tile = darm.plan_info(dtype_code, n, has_vals, "melded")
    per_kind = {}
    for _ in range(args.steps):
        reset()
        for name, t in darm.sort_profile(work_k, work_v, variant="melded"):
            per_kind.setdefault(name, []).append(t)
    totals = {k: sum(v) for k, v in per_kind.items()}
    dom = max(totals, key=totals.get)
    avg_ms = statistics.mean(per_kind[dom])
    bytes_per_launch = 2 * n * elem_bytes  # each pass reads and writes the array once
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    peak = None
    peak_src = "measured"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        peak = 6800.0
        peak_src = "fallback"
    whole_sort_gbs = bytes_per_launch * passes / (ms_meld / args.steps * 1e-3) / 1e9

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        hk = torch.empty(n, dtype=src_k.dtype, pin_memory=True).numpy()
        hv = torch.empty(n, dtype=torch.uint32, pin_memory=True).numpy() if has_vals else None
        for _ in range(2):
            hk[:] = keys_np
            if has_vals:
                hv[:] = vals_np
            darm.sort_host(hk, hv, variant="melded")
        tot = 0.0
        for _ in range(args.steps):
            hk[:] = keys_np
            if has_vals:
                hv[:] = vals_np
            t0 = time.perf_counter()
            darm.sort_host(hk, hv, variant="melded")
            tot += time.perf_counter() - t0
        tot = max_over_ranks(tot, world)
        e2e = {"value": world * n * args.steps / tot, "unit": "keys/s",
               "h2d_bytes_per_step": n * elem_bytes, "d2h_bytes_per_step": n * elem_bytes}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_meld / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if keys_np.dtype == np.float32 else "u32",
            "data": "synthetic",
            "config": {"workload": desc, "n": n, "variant": "melded",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "hbm_passes": passes, "tile": tile},
            "divergent": {"value": value_div, "ms_per_step": ms_div / args.steps},
            "melded_over_divergent": value / value_div,
            "roofline": {"bound": "hbm" if passes > 1 else "latency",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": recorded_traffic(args.workload, dom),
                         "algorithmic_bytes": bytes_per_launch, "kernel": f"{dom} pass",
                         "peak_source": peak_src,
                         "whole_sort_gbs": whole_sort_gbs,
                         "whole_sort_frac": whole_sort_gbs / peak,
                         "pass_ms": {k: statistics.mean(v) for k, v in per_kind.items()},
                         "pass_share": {k: totals[k] / sum(totals.values()) for k in totals},
                         "pass_timing": "each launch of the array's plan timed alone with CUDA "
                                        "events on its stream (plan order, whole-array launches); "
                                        "the timed sorts of 2^22 elements or more run the two "
                                        "halves' passes concurrently on two streams",
                         **({"note": "one tile on one SM: every stage in one launch, bound "
                                     "by latency, not by HBM"} if passes == 1 else {})},
            "clocks": clk,
            "gpu_launches": launches_meld + launches_div,
        }
        if e2e is not None:
            line["e2e"] = e2e
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(keys_np, vals_np)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
