"""Benchmark: vqsort on GB300, one JSON line on stdout.

Workload: one array of 1e8 uniform random uint64 keys (full 64-bit range,
seeded SplitMix64), sorted ascending by the plain path; a step is one full
sort (all partition levels, leaves, fallback check). Inputs are 800 MB per
array, larger than L2, and every timed step sorts its own fresh copy, so no
step sees a cache warmed by the previous one.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--n N_KEYS] [--dtype u64] [--dist uniform]

--impl reference times the CPU oracle (plain scalar Quicksort) on host cores
instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2205_05982_gb300 import inputs  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
# sources of the partition and leaf kernels: a recorded DRAM traffic figure
# is used only while these files are unchanged since the capture
KERNEL_SOURCES = ("paper_2205_05982_gb300/csrc/partition.cu", "paper_2205_05982_gb300/csrc/common.cuh",
                  "paper_2205_05982_gb300/csrc/launch.h")
LEAF_SOURCES = ("paper_2205_05982_gb300/csrc/leaf.cu", "paper_2205_05982_gb300/csrc/sortnet.cuh",
                "paper_2205_05982_gb300/csrc/networks.h", "paper_2205_05982_gb300/csrc/common.cuh",
                "paper_2205_05982_gb300/csrc/launch.h")


def kernel_hash(sources=KERNEL_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(key: str, sources) -> int | None:
    """DRAM bytes per launch recorded in profiles/traffic.json for `key`, if
    the kernel's sources still hash to the captured build."""
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if key in tr and tr[key].get("kernel_hash") == kernel_hash(sources):
            return tr[key]["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        pass
    return None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=100_000_000)
    p.add_argument("--dtype", default="u64")
    p.add_argument("--dist", default="uniform")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--e2e-steps", type=int, default=6)
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline (profiling runs)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the per-dtype, batched and served measurements")
    p.add_argument("--served-requests", type=int, default=10_000)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


METRIC = "sort throughput (GKeys/s), 1e8 keys per array"


def partition_bytes(kb: int, st: dict) -> int:
    """Algorithmic bytes of one partition launch: every partitioned key is
    read and written once (two-way and K-way scatter passes), and K-way
    ranges read their keys once more in the counting pass."""
    return kb * (2 * st["keys_partitioned"] + st["keys_counted"])


# Integer lane operations of one compare-exchange of two codes: 32-bit codes
# (2- and 4-byte keys) take a min and a max; 64-bit codes a two-word compare
# and four selects; 128-bit codes a four-word compare chain and eight selects.
ALU_OPS_PER_CE = {2: 2, 4: 2, 8: 6, 16: 13}


def alu_peak(clk):
    """Lane operations per second of the integer ALU pipes: SMs x 4 SM
    sub-partitions x 16 ALU lanes (ncu shows the ALU pipe busier than the
    issue slots, i.e. a half-rate pipe) x the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    return sms * 4 * 16 * mhz * 1e6, f"derived: {sms} SMs x 4 sub-partitions x 16 ALU lanes x {mhz:.0f} MHz"


# Nominal HBM3e bandwidth of one GB300 (the measured copy bandwidth is the
# main denominator; this one is reported beside it).
NOMINAL_HBM_GBS = 8000.0
# Leaf cutoff the library uses by key size when none is set.
DEFAULT_LEAF_CUTOFF = {2: 4096, 4: 4096, 8: 8192, 16: 4096}


def ideal_two_way(kb: int, n: int, cutoff: int) -> dict:
    """Bytes of an ideal two-way Quicksort of n keys: every level halves every
    range exactly, so ceil(log2(n / cutoff)) partition levels and one leaf
    pass each read and write all n keys. A bad pivot cannot inflate the
    fraction measured against this (the levels are not the ones run), and
    K-way levels can beat it."""
    levels = max(0, math.ceil(math.log2(n / cutoff))) if n > cutoff else 0
    return {"bytes": 2 * n * kb * (levels + 1), "partition_levels": levels, "leaf_cutoff": cutoff}


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return FALLBACK_HBM_GBS, "fallback"


def workload(args):
    return {
        "workload": f"{args.n:.0e} {args.dist} {args.dtype} keys, one array, ascending "
                    "(plain partition + sorting-network Quicksort)",
        "n_keys": args.n, "key_type": args.dtype, "distribution": args.dist,
        "seed": inputs.DEFAULT_SEED,
        "l2": "inputs larger than L2 (one fresh array per timed step)",
    }


def make_input(args):
    if args.dtype == "kv64":
        return inputs.kv_pairs(args.n)
    return inputs.make(args.dtype, args.n, args.dist, specials=args.dtype in ("f32", "f64"))


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, single thread, bounded sample.
# ---------------------------------------------------------------------------

def cpu_baseline(args, a, seconds):
    import oracle
    oracle.build()
    sample_n = min(len(a), 10_000_000)
    sample = a[:sample_n]
    times = []
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        oracle.sort(sample, args.dtype, True)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or len(times) >= 10:
            break
    med = statistics.median(times)
    return {
        "value": sample_n / med / 1e9, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
        "sample": f"first {sample_n:.0e} keys of the same array, sorted {len(times)} times "
                  f"(median {med:.2f} s); scalar median-of-3 Quicksort, 1 thread",
    }


# Keys per second the oracle sorts on one Grace core (u64, 1e7 keys: 0.016
# GKeys/s); sizes the reference arm's per-step sample so that its warm-up and
# timed steps together take about REFERENCE_SECONDS.
ORACLE_KEYS_PER_S = 16e6
REFERENCE_SECONDS = 90.0


def reference_sample_keys(n: int, steps: int, warmup: int) -> int:
    """Keys per step of the reference arm: the whole run stays near
    REFERENCE_SECONDS, at most 1e7 keys and at least 1e5 (or n)."""
    per_step = REFERENCE_SECONDS * ORACLE_KEYS_PER_S / max(1, steps + warmup)
    return int(min(n, 10_000_000, max(100_000, per_step)))


def run_reference(args):
    """The oracle as it stands, on one host core: `warmup` untimed and
    `steps` timed sorts of a bounded sample of the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    a = make_input(args)
    sample_n = reference_sample_keys(len(a), args.steps, args.warmup)
    sample = a[:sample_n]
    for _ in range(args.warmup):
        oracle.sort(sample, args.dtype, True)
    times = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        oracle.sort(sample, args.dtype, True)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample_n * len(times) / total / 1e9
    cb = {"value": value, "unit": "GKeys/s", "cores": 1, "kind": "oracle",
          "sample": f"first {sample_n:.0e} keys of the same array per step, {len(times)} timed steps "
                    f"after {args.warmup} untimed ({total:.2f} s timed); scalar median-of-3 Quicksort "
                    f"with the Heapsort depth bound, 1 thread"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "GKeys/s", "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup,
        "ms_per_step": total / len(times) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.dtype,
        "data": "synthetic", "config": workload(args), "cpu_baseline": cb,
        "e2e": {"value": value, "unit": "GKeys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:  # noqa: BLE001
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm.
# ---------------------------------------------------------------------------

def max_over_ranks(value: float, dist=None) -> float:
    """The slowest rank's time: every rank gets the maximum (any backend)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def to_device_bits(a, dtype, torch):
    view = {2: np.int16, 4: np.int32, 8: np.int64, 16: np.int64}[inputs.KEY_BYTES[dtype]]
    host = a if dtype in ("f32", "f64") else a.view(view)
    return torch.from_numpy(np.ascontiguousarray(host)).cuda()


def bits_view(t, torch):
    """The same memory as an integer tensor of the same element width."""
    return t.view({2: torch.int16, 4: torch.int32, 8: torch.int64}[t.element_size()])


def time_sorts(vq, torch, copies, ws, dtype, warmup, descending=False):
    """Sorts copies[0:warmup] untimed, then each remaining copy; returns
    (ms per sort, stats of the last sort, per-kernel profile)."""
    for i in range(warmup):
        vq.sort_ws_(copies[i], ws, dtype, descending=descending)
    torch.cuda.synchronize()
    vq.profile_reset()
    vq.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for c in copies[warmup:]:
        vq.sort_ws_(c, ws, dtype, descending=descending)
    e1.record()
    torch.cuda.synchronize()
    vq.profile_enable(False)
    prof = vq.profile_read()
    st = vq.stats(ws)
    return e0.elapsed_time(e1) / (len(copies) - warmup), st, prof


def extra_dtypes(vq, torch, peak, n):
    """The other key types of the 1e8-keys-per-dtype workload (uniform)."""
    out = {}
    for dt in ("f32", "i32", "i16"):
        a = inputs.make(dt, n, "uniform", specials=dt == "f32")
        src = to_device_bits(a, dt, torch)
        copies = [src.clone() for _ in range(4)]
        ws = vq.alloc_workspace(dt, n)
        ms, st, prof = time_sorts(vq, torch, copies, ws, dt, 1)
        kb = inputs.KEY_BYTES[dt]
        part = prof.get("partition", {"ms": float("nan"), "launches": 1})
        part_ms = part["ms"] / max(1, part["launches"])
        pb = partition_bytes(kb, st)
        out[dt] = {"gkeys_per_s": n / (ms * 1e-3) / 1e9, "ms": ms,
                   "partition_frac": pb / (part_ms * 1e-3) / 1e9 / peak,
                   "sort_frac": (pb + 2 * kb * n) / (ms * 1e-3) / 1e9 / peak,
                   "max_depth": st["max_depth"]}
        del copies, src, ws
        torch.cuda.empty_cache()
    return out


DISTRIBUTIONS = ("uniform", "distinct16", "equal", "sorted", "reverse", "organpipe")


def extra_distributions(vq, torch, n):
    """The 48 runs of the 1e8-keys-per-dtype workload: u64, f32, i32 and i16
    keys in six distributions (uniform, 16 distinct values, all equal,
    sorted, reverse sorted, organ pipe), each sorted ascending and
    descending; GKeys/s over two timed sorts after one warm-up."""
    out = {}
    for dt in ("u64", "f32", "i32", "i16"):
        ws = vq.alloc_workspace(dt, n)
        srt = None
        for dist in DISTRIBUTIONS:
            if dist == "reverse":   # the sorted array backwards (as the generator makes it)
                src = torch.flip(srt, [0]).contiguous()
                srt = None
            else:
                src = to_device_bits(inputs.make(dt, n, dist, specials=dt == "f32"), dt, torch)
                if dist == "sorted":
                    srt = src.clone()
            for desc in (False, True):
                copies = [src.clone() for _ in range(3)]
                ms, st, _ = time_sorts(vq, torch, copies, ws, dt, 1, descending=desc)
                assert st["device_status"] == 0, (dt, dist, desc, st)
                out[f"{dt}:{dist}:{'desc' if desc else 'asc'}"] = {
                    "gkeys_per_s": n / (ms * 1e-3) / 1e9, "ms": ms, "max_depth": st["max_depth"],
                    "fallback_keys": st["fallback_keys"], "equal_keys": st["equal_keys"]}
                del copies
            del src
        del ws
        torch.cuda.empty_cache()
    return out


def extra_wide(vq, torch, peak, n=25_000_000):
    """Wide keys: 2.5e7 u128 keys (two uniform halves) and 2.5e7 kv64 pairs
    (uniform key, value = index, 10 % of keys duplicated)."""
    out = {}
    for dt in ("u128", "kv64"):
        a = inputs.kv_pairs(n) if dt == "kv64" else inputs.make(dt, n, "uniform")
        src = to_device_bits(a, dt, torch)
        copies = [src.clone() for _ in range(4)]
        ws = vq.alloc_workspace(dt, n)
        ms, st, prof = time_sorts(vq, torch, copies, ws, dt, 1)
        part = prof.get("partition", {"ms": float("nan"), "launches": 1})
        part_ms = part["ms"] / max(1, part["launches"])
        out[dt] = {"gkeys_per_s": n / (ms * 1e-3) / 1e9, "ms": ms,
                   "partition_frac": partition_bytes(16, st) / (part_ms * 1e-3) / 1e9 / peak,
                   "leaf_ms": sum(v["ms"] for k, v in prof.items() if k.startswith("leaf")) / max(1, part["launches"])}
        del copies, src, ws
        torch.cuda.empty_cache()
    return out


def extra_stable(vq, torch, n, reps=5):
    """Stable sorts (Sec. 5 row-id recipe) of n uniform keys: keys of up to 4
    bytes travel as 64-bit (code, row) codes, 8-byte keys as 128-bit ones."""
    res = {}
    for dt in ("u32", "u64"):
        a = inputs.make(dt, n, "uniform")
        src = to_device_bits(a, dt, torch)
        t = src.clone()
        for _ in range(2):
            t.copy_(src)
            vq.sort_stable_(t, dt)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            t.copy_(src)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            vq.sort_stable_(t, dt)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = float(np.median(ms))
        res[dt] = {"gkeys_per_s": n / (m * 1e-3) / 1e9, "ms": m}
        del src, t
        torch.cuda.empty_cache()
    return res


def extra_partition_sweep(vq, torch, peak, reps=10):
    """One Partition (Sec. 2.1) on its own: 2^24 doubles (the paper's
    partition microbenchmark) and a sweep of sizes and key types. Each call
    partitions n uniform keys around the key at n/2 into a second buffer.
    `kernel_gbs` is the algorithmic traffic (2 x key bytes x n) over the
    partition kernel's own time; `call_gbs` over the whole call (counter
    reset, pivot setup and partition kernel, back to back)."""
    res = {}
    for dt in ("f64", "u64", "f32", "u32", "i16", "u128"):
        kb = inputs.KEY_BYTES[dt]
        for lg in (16, 18, 20, 22, 24, 26):
            n = 1 << lg
            a = inputs.make(dt, n, "uniform", seed=lg)
            src = to_device_bits(a, dt, torch)
            piv = a[n // 2]
            for _ in range(3):
                vq.partition(src, piv, dt)
            torch.cuda.synchronize()
            vq.profile_reset()
            vq.profile_enable(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                vq.partition(src, piv, dt)
            e1.record()
            torch.cuda.synchronize()
            vq.profile_enable(False)
            prof = vq.profile_read()
            call_ms = e0.elapsed_time(e1) / reps
            pk = prof.get("partition", {"ms": float("nan"), "launches": 1})
            kern_ms = pk["ms"] / max(1, pk["launches"])
            byts = 2 * kb * n
            res[f"{dt}:2^{lg}"] = {"kernel_ms": kern_ms, "kernel_gbs": byts / (kern_ms * 1e-3) / 1e9,
                                   "kernel_frac": byts / (kern_ms * 1e-3) / 1e9 / peak,
                                   "call_ms": call_ms, "call_gbs": byts / (call_ms * 1e-3) / 1e9}
            del src
    torch.cuda.empty_cache()
    return res


def extra_batched(vq, torch, reps=5):
    """16,384 arrays, sizes log-uniform in [16, 65536], uniform u32 keys:
    one autotuned segmented sort replayed as a CUDA graph vs one plain sort
    launch set per array. Outputs are compared byte for byte."""
    from paper_2205_05982_gb300 import batch
    res = {}
    for dt in ("u32", "f32"):
        sizes = inputs.segment_sizes(16384, 16, 65536)
        off = inputs.offsets_from_sizes(sizes)
        n = int(off[-1])
        a = inputs.make(dt, n, "uniform", seed=7, specials=dt == "f32")
        src = to_device_bits(a, dt, torch)
        tune = batch.autotune(src.clone(), off, dt, reps=2)
        b = batch.SegmentedBatch(src.clone(), off, dt, settings=tune["settings"])
        b.capture()
        g_ms = []
        for _ in range(reps):
            b.keys.copy_(src)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            with torch.cuda.stream(b.stream):
                b.graph.replay()
            e1.record(b.stream)
            torch.cuda.synchronize()
            g_ms.append(e0.elapsed_time(e1))
        graph_out = b.keys.clone()
        each = src.clone()
        ws1 = vq.alloc_workspace(dt, int(sizes.max()), 1)
        p_ms = []
        for _ in range(max(1, reps // 2)):
            each.copy_(src)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.sort_each(each, off, dt, ws=ws1)
            e1.record()
            torch.cuda.synchronize()
            p_ms.append(e0.elapsed_time(e1))
        # bit patterns (f32 holds NaNs, which never compare equal as floats)
        same = bool(torch.equal(bits_view(graph_out, torch), bits_view(each, torch)))
        gm, pm = float(np.median(g_ms)), float(np.median(p_ms))
        res[dt] = {"arrays": int(sizes.size), "keys": n, "graph_ms": gm, "per_array_ms": pm,
                   "graph_gkeys_per_s": n / (gm * 1e-3) / 1e9,
                   "per_array_gkeys_per_s": n / (pm * 1e-3) / 1e9, "speedup": pm / gm,
                   "identical_output": same, "tuned": tune["settings"],
                   "tuned_ms": tune["ms"], "default_ms": tune["default_ms"]}
        del b, src, each
        torch.cuda.empty_cache()
    return res


def extra_served(vq, torch, num):
    """Poisson stream of `num` requests, sizes log-uniform in [1e3, 1e7],
    key type uniform over {i16, u32, f32, u64, kv64}, admitted under a 40 GB
    budget: saturated capacity, then arrivals at 0.8 x capacity served with
    continuous batching (8 slots) and one at a time (plain)."""
    from paper_2205_05982_gb300 import serve
    hi = 10_000_000
    sources = {}
    for dt in ("i16", "u32", "f32", "u64"):
        sources[dt] = to_device_bits(inputs.make(dt, hi, "uniform", seed=3, specials=dt == "f32"), dt, torch)
    sources["kv64"] = to_device_bits(inputs.kv_pairs(hi, seed=3), "kv64", torch)
    server = serve.Server(slots=8, budget_bytes=40 * 10**9, max_keys=hi)
    burst = serve.poisson_requests(num, 1e12, sources, seed=5)      # all arrive at once
    sat = server.run(burst)
    rate = 0.8 * sat["requests"] / (sat["span_ms"] * 1e-3)
    reqs = serve.poisson_requests(num, rate, sources, seed=6)
    served = server.run(reqs)
    plain = serve.run_plain(serve.poisson_requests(num, rate, sources, seed=6), max_keys=hi)
    del server, sources
    torch.cuda.empty_cache()
    return {"requests": num, "rate_per_s": rate, "saturated": sat, "served": served, "plain": plain,
            "p99_speedup": plain["p99_ms"] / served["p99_ms"],
            "throughput_ratio": served["gkeys_per_s"] / plain["gkeys_per_s"]}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_2205_05982_gb300 as vq

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vq.load()
    kb = inputs.KEY_BYTES[args.dtype]

    a = make_input(args)
    src = to_device_bits(a, args.dtype, torch)
    copies = [src.clone() for _ in range(args.steps + args.warmup)]
    ws = vq.alloc_workspace(args.dtype, args.n)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    for i in range(args.warmup):
        vq.sort_ws_(copies[i], ws, args.dtype)
    torch.cuda.synchronize()
    st = vq.stats(ws)
    assert st["device_status"] == 0, st

    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    vq.profile_reset()
    vq.profile_enable(True)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        vq.sort_ws_(copies[args.warmup + i], ws, args.dtype)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    vq.profile_enable(False)
    prof = vq.profile_read()
    ms_total = e0.elapsed_time(e1)
    st = vq.stats(ws)
    assert st["device_status"] == 0, st
    ms_total = max_over_ranks(ms_total, dist if world > 1 else None)
    ms_step = ms_total / args.steps

    # spot check: the last timed output is sorted (codes non-decreasing)
    out = copies[-1]
    if args.dtype == "u64":
        enc = out ^ torch.tensor(-2 ** 63, dtype=torch.int64, device=out.device)
        assert bool((enc[1:] >= enc[:-1]).all())
    del copies

    # roofline of the dominant kernel (the persistent partition kernel)
    part = prof.get("partition", {"ms": float("nan"), "launches": 1})
    part_ms = part["ms"] / max(1, part["launches"])
    part_bytes = partition_bytes(kb, st)
    peak, peak_kind = hbm_peak()
    achieved = part_bytes / (part_ms * 1e-3) / 1e9
    traffic = recorded_traffic(f"{args.dtype}:{args.n}:{args.dist}", KERNEL_SOURCES)
    leaf_ms = sum(v["ms"] for k, v in prof.items() if k.startswith("leaf")) / args.steps
    sort_bytes = part_bytes + 2 * kb * args.n
    ideal = ideal_two_way(kb, args.n, vq.get_option("leaf_cutoff") or DEFAULT_LEAF_CUTOFF[kb])
    kernels = {k: {"ms_per_launch": v["ms"] / max(1, v["launches"]), "launches": v["launches"]}
               for k, v in prof.items()}
    gpu_launches = sum(v["launches"] for v in prof.values())

    # end to end through the public host-buffer API: every step uploads its
    # own pinned array, sorts it and brings the keys back into it; steps
    # alternate between two streams (vqsort_sort_host_async), so one array
    # uploads while the other sorts and writes back over the other direction
    # of the host link. The single synchronous call is reported beside it.
    e2e_val = e2e_single = e2e_link = None
    if not args.no_e2e:
        steps = max(2, args.e2e_steps)
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        bufs, views = [], []
        for _ in range(steps):
            buf = torch.empty(src.numel() * src.element_size(), dtype=torch.uint8, pin_memory=True)
            v = buf.numpy().view(a.dtype).reshape(a.shape)
            v[...] = a
            bufs.append(buf)
            views.append(v)
        for i in range(2):   # each stream's device copy and workspace, full size (untimed)
            vq.sort_host_async(views[i], args.dtype, stream=streams[i])
        for st_ in streams:
            st_.synchronize()
        views[0][...] = a
        views[1][...] = a
        t0 = time.perf_counter()
        for i in range(steps):
            vq.sort_host_async(views[i], args.dtype, stream=streams[i % 2])
        for st_ in streams:
            st_.synchronize()
        t_pipe = time.perf_counter() - t0
        for st_ in streams:
            assert vq.last_device_status(None, st_) == 0
        if args.dtype == "u64":
            tail = views[-1][: 1 << 20]
            assert bool((tail[1:] >= tail[:-1]).all())
        e2e_val = world * args.n * steps / t_pipe / 1e9
        views[0][...] = a
        t0 = time.perf_counter()
        vq.sort_host(views[0], args.dtype)
        e2e_single = world * args.n / (time.perf_counter() - t0) / 1e9
        # the host link of this machine (plain pinned copies of the same size,
        # best of three), to read the end-to-end numbers against
        dev = torch.empty(bufs[0].numel(), dtype=torch.uint8, device=f"cuda:{local}")

        def copy_ms(dst, srcb):
            best = float("inf")
            for _ in range(3):
                c0 = torch.cuda.Event(enable_timing=True)
                c1 = torch.cuda.Event(enable_timing=True)
                c0.record()
                dst.copy_(srcb, non_blocking=True)
                c1.record()
                c1.synchronize()
                best = min(best, c0.elapsed_time(c1))
            return best

        # every array of the timed loop: host sorts of different pinned
        # arrays of one process were measured at very different rates
        h2d_ms = [copy_ms(dev, b) for b in bufs]
        d2h_ms = [copy_ms(b, dev) for b in bufs]
        nbytes = bufs[0].numel()
        h2d_med, d2h_med = statistics.median(h2d_ms), statistics.median(d2h_ms)
        e2e_link = {"h2d_gbs": nbytes / h2d_med / 1e6, "d2h_gbs": nbytes / d2h_med / 1e6,
                    "copy_only_gkeys_per_s": args.n / ((h2d_med + d2h_med) * 1e-3) / 1e9,
                    "per_array_h2d_gbs": [round(nbytes / t / 1e6, 1) for t in h2d_ms],
                    "per_array_d2h_gbs": [round(nbytes / t / 1e6, 1) for t in d2h_ms],
                    "how": "each pinned array of the timed loop up, then down, no sort (CUDA events, "
                           "best of 3 per array; the scalar rates are the medians)"}
        del dev, bufs, views

    line = {
        "metric": METRIC,
        "value": world * args.n / (ms_step * 1e-3) / 1e9,
        "unit": "GKeys/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": workload(args),
        "roofline": None,   # the dominant kernel's, set below
        "roofline_partition": {"bound": "hbm", "kernel": "k_partition (persistent partition levels)",
                               "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                               "algorithmic_bytes_per_launch": part_bytes},
        "sort_roofline": {"bytes_per_step": sort_bytes,
                          "achieved_gbs": sort_bytes / (ms_step * 1e-3) / 1e9,
                          "frac": sort_bytes / (ms_step * 1e-3) / 1e9 / peak,
                          "frac_nominal": sort_bytes / (ms_step * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
                          "ideal_two_way": dict(ideal, ms_at_peak=ideal["bytes"] / peak / 1e6,
                                                frac=ideal["bytes"] / peak / 1e6 / ms_step,
                                                frac_nominal=ideal["bytes"] / NOMINAL_HBM_GBS / 1e6 / ms_step),
                          "levels_run_keys": st["keys_partitioned"], "keys_counted": st["keys_counted"],
                          "kway_ranges": st["kway_ranges"], "max_depth": st["max_depth"],
                          "leaf_ms_per_step": leaf_ms},
        "kernels": kernels,
        "kernel_hash": kernel_hash(),
        "gpu_launches": gpu_launches,
        "e2e": {"value": e2e_val, "unit": "GKeys/s", "h2d_bytes_per_step": args.n * kb,
                "d2h_bytes_per_step": args.n * kb,
                "path": "vqsort_sort_host_async, one pinned host array per step, steps alternating over two "
                        "streams (upload, sort and write-back of every step inside the timed region)",
                "single_call": e2e_single, "single_call_path": "vqsort_sort_host (one array, waits)",
                "link": e2e_link},
        "clocks": clk,
    }
    # the leaf networks: compare-exchanges (counted on the device) x integer
    # operations per compare-exchange, over the leaf kernels' time
    apeak, apeak_kind = alu_peak(clk)
    ce = st["leaf_ce"]
    leaf_ops = ce * ALU_OPS_PER_CE[kb]
    leaf_achieved = leaf_ops / (leaf_ms * 1e-3) if leaf_ms > 0 else 0.0
    line["roofline_leaf"] = {"bound": "alu", "kernel": "k_leaf_warp + k_leaf_mid + k_leaf_block (sorting networks)",
                             "achieved": leaf_achieved / 1e12, "peak": apeak / 1e12, "unit": "Tlane-op/s",
                             "frac": leaf_achieved / apeak, "peak_source": apeak_kind,
                             "traffic": recorded_traffic(f"leaf:{args.dtype}:{args.n}:{args.dist}", LEAF_SOURCES),
                             "compare_exchanges_per_step": ce, "ops_per_compare_exchange": ALU_OPS_PER_CE[kb]}
    # the dominant kernel by measured time decides which one is "roofline"
    line["roofline"] = dict(line["roofline_leaf"] if leaf_ms > part_ms else line["roofline_partition"])
    if rank == 0:
        if not args.no_extras:
            del src
            torch.cuda.empty_cache()
            line["per_dtype"] = extra_dtypes(vq, torch, peak, args.n)
            line["distributions"] = extra_distributions(vq, torch, args.n)
            line["wide"] = extra_wide(vq, torch, peak)
            line["partition_sweep"] = extra_partition_sweep(vq, torch, peak)
            line["stable"] = extra_stable(vq, torch, args.n)
            line["batched"] = extra_batched(vq, torch)
            line["served"] = extra_served(vq, torch, args.served_requests)
        line["cpu_baseline"] = None if args.no_cpu else cpu_baseline(args, a, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
