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


def recorded_traffic(key: str, sources, field: str = "bytes_per_launch") -> int | None:
    """A per-launch ncu figure recorded in profiles/traffic.json for `key`
    (DRAM bytes, or warp instructions with field="inst_per_launch"), if the
    kernel's sources still hash to the captured build."""
    try:
        with open(TRAFFIC_FILE) as f:
            tr = json.load(f)
        if key in tr and tr[key].get("kernel_hash") == kernel_hash(sources):
            return tr[key].get(field)
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
    p.add_argument("--leaf-cutoff", type=int, default=0,
                   help="leaf cutoff option (0: the library's rule for the array length); lets a profiling "
                        "run of a smaller array keep the partition levels of a larger one")
    p.add_argument("--leaf-sizes", default=None,
                   help="LO,HI: leaf microbenchmark instead: --n keys in segments of LO..HI keys (each at most "
                        "the leaf cutoff, so every segment goes straight to a leaf kernel)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


METRIC = "sort throughput (GKeys/s), 1e8 keys per array"


def partition_bytes(kb: int, st: dict) -> int:
    """Algorithmic bytes of one partition launch: every key of every range
    partitioned at a level is read once and written once (2 x key bytes per
    key and level, two-way and K-way levels alike)."""
    return 2 * kb * st["keys_partitioned"]


def partition_overhead_bytes(kb: int, st: dict) -> dict:
    """Bytes the K-way levels move beyond the algorithmic ones: the counting
    pass reads every key once more, and each key's bucket byte is written by
    the counting pass and read back by the scatter pass."""
    return {"counting_reread": kb * st["keys_counted"], "bucket_bytes": 2 * st["keys_counted"]}


def leaf_bytes(kb: int, st: dict, kernel: str) -> int:
    """Algorithmic bytes of one leaf launch: each key of its ranges is read
    once and written once; the block leaf kernel also copies the all-equal
    ranges."""
    keys = {"leaf_warp": st["leaf_keys_warp"], "leaf_mid": st["leaf_keys_mid"],
            "leaf_block": st["leaf_keys_block"] + st["equal_keys"]}[kernel]
    return 2 * kb * keys


def issue_peak():
    """Measured integer ALU-pipe rate of this GPU: the library's throughput
    probe (eight independent 32-bit min + xor chains per thread, 8 blocks of
    256 threads per SM; both instructions run on the ALU pipe), one warp
    instruction per 32 lane operations."""
    import paper_2205_05982_gb300 as vq
    p = vq.probe_int_throughput(kind=0)
    p64 = vq.probe_int_throughput(kind=1)
    return {"warp_inst_per_s": p["lane_ops_per_s"] / 32, "lane_ops_per_s": p["lane_ops_per_s"],
            "min64_per_s": p64["lane_ops_per_s"] / 6,
            "how": "vqsort_probe_int_throughput kind 0 (32-bit min + xor, 2 lane ops) and kind 1 (64-bit "
                   "compare + 2 selects + xor, 6 lane ops), CUDA events, best of 5; loop overhead uncounted"}


# Nominal HBM3e bandwidth of one GB300 (the measured copy bandwidth is the
# main denominator; this one is reported beside it).
NOMINAL_HBM_GBS = 8000.0
# Leaf cutoff the library uses by key size when none is set, for large
# arrays and segmented batches.
DEFAULT_LEAF_CUTOFF = {2: 4096, 4: 4096, 8: 4096, 16: 4096}
# The library's size rule for one array of n keys (launch.h size_leaf_cutoff):
# 16384 up to the small bound, 8192 below the mid bound.
LEAF_N_SMALL = {"wide": 1 << 21, "narrow": 1 << 22}
LEAF_N_MID = {"wide": 1 << 26, "narrow": 1 << 25}


def default_leaf_cutoff(kb: int, n: int, segments: int = 1) -> int:
    if segments != 1 or kb == 16:
        return DEFAULT_LEAF_CUTOFF[kb]
    w = "wide" if kb == 8 else "narrow"
    return 16384 if n <= LEAF_N_SMALL[w] else 8192 if n < LEAF_N_MID[w] else DEFAULT_LEAF_CUTOFF[kb]


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
        "leaf_cutoff": getattr(args, "leaf_cutoff", 0) or default_leaf_cutoff(inputs.KEY_BYTES[args.dtype], args.n),
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


def order_codes(t, dtype, torch):
    """Signed integers whose order is the sort order of the keys in t (same
    bit patterns; IEEE totalOrder for floats): the check below compares these
    with torch's own operators. Unsigned keys flip the sign bit; negative
    floats flip every bit but the sign."""
    b = bits_view(t.reshape(-1), torch) if dtype not in ("u128", "kv64") else None
    if dtype in ("u16", "u32", "u64"):
        return b ^ torch.iinfo(b.dtype).min
    if dtype in ("f32", "f64"):
        return b ^ ((b >> (8 * b.element_size() - 1)) & torch.iinfo(b.dtype).max)
    return b


def check_sorted_permutation(out, src, dtype, descending, torch) -> bool:
    """The output is ordered (codes non-decreasing, or non-increasing when
    descending) and holds the input's bit patterns as a multiset (equal
    after sorting both as plain integers with torch.sort)."""
    if inputs.KEY_BYTES[dtype] == 16:
        raise ValueError("16-byte keys are checked by the tests")
    c = order_codes(out, dtype, torch)
    ok = bool((c[1:] <= c[:-1]).all()) if descending else bool((c[1:] >= c[:-1]).all())
    bo, bs = bits_view(out.reshape(-1), torch), bits_view(src.reshape(-1), torch)
    return ok and bool(torch.equal(torch.sort(bo).values, torch.sort(bs).values))


def time_sorts(vq, torch, copies, ws, dtype, warmup, descending=False, by_key=False):
    """Sorts copies[0:warmup] untimed, then each remaining copy; returns
    (ms per sort, stats of the last sort, per-kernel profile). by_key: kv64
    pairs in the key-only order (vqsort_sort_kv_by_key_ws)."""
    def one(c):
        if by_key:
            vq.sort_kv_by_key_(c, descending=descending, ws=ws)
        else:
            vq.sort_ws_(c, ws, dtype, descending=descending)
    for i in range(warmup):
        one(copies[i])
    torch.cuda.synchronize()
    vq.profile_reset()
    vq.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for c in copies[warmup:]:
        one(c)
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


def extra_c1(vq, torch, reps=20):
    """One array of 1e6 uniform u64 keys, ascending, plain path. The array
    (8 MB) fits in L2, so a 256 MB buffer is written between timed sorts
    (outside the timed region) and every sort starts from HBM."""
    n = 1_000_000
    a = inputs.make("u64", n, "uniform")
    src = to_device_bits(a, "u64", torch)
    t = src.clone()
    ws = vq.alloc_workspace("u64", n)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=src.device)
    for _ in range(3):
        t.copy_(src)
        vq.sort_ws_(t, ws, "u64")
    torch.cuda.synchronize()
    ms = []
    for i in range(reps):
        t.copy_(src)
        flush.fill_(i & 255)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        vq.sort_ws_(t, ws, "u64")
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    st = vq.stats(ws)
    assert st["device_status"] == 0, st
    assert check_sorted_permutation(t, src, "u64", False, torch)
    med = statistics.median(ms)
    res = {"workload": "1e6 uniform u64 keys, one array, ascending (plain path)", "n_keys": n,
           "gkeys_per_s": n / (med * 1e-3) / 1e9, "us_per_sort": med * 1e3,
           "us_p10": float(np.percentile(ms, 10)) * 1e3, "us_p90": float(np.percentile(ms, 90)) * 1e3,
           "sorts": reps, "l2": "256 MB written between timed sorts", "launches_per_sort": 7,
           "leaf_cutoff": default_leaf_cutoff(8, n),
           "max_depth": st["max_depth"], "kway_ranges": st["kway_ranges"]}
    del t, src, ws, flush
    torch.cuda.empty_cache()
    return res


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
                # every timed output: ordered, and a permutation of the input
                for c in copies:
                    assert check_sorted_permutation(c, src, dt, desc, torch), (dt, dist, desc)
                out[f"{dt}:{dist}:{'desc' if desc else 'asc'}"] = {
                    "gkeys_per_s": n / (ms * 1e-3) / 1e9, "ms": ms, "max_depth": st["max_depth"],
                    "fallback_keys": st["fallback_keys"], "equal_keys": st["equal_keys"],
                    "outputs_checked": len(copies)}
                del copies
            del src
        del ws
        torch.cuda.empty_cache()
    return out


def extra_wide(vq, torch, peak, n=25_000_000):
    """Wide keys: 2.5e7 u128 keys (two uniform halves) and 2.5e7 kv64 pairs
    (uniform key, value = index, 10 % of keys duplicated)."""
    out = {}
    for dt in ("u128", "kv64", "kv64_by_key"):
        a = inputs.kv_pairs(n) if dt.startswith("kv64") else inputs.make(dt, n, "uniform")
        src = to_device_bits(a, "kv64" if dt.startswith("kv64") else dt, torch)
        copies = [src.clone() for _ in range(4)]
        ws = vq.alloc_workspace("kv64" if dt.startswith("kv64") else dt, n)
        ms, st, prof = time_sorts(vq, torch, copies, ws, dt[:4], 1, by_key=dt == "kv64_by_key")
        if dt == "kv64_by_key":   # keys ordered, every value beside its key (value = index)
            k = copies[-1][:, 0]
            kc = k ^ torch.iinfo(torch.int64).min
            assert bool((kc[1:] >= kc[:-1]).all())
            assert bool(torch.equal(k, src[copies[-1][:, 1], 0]))
            assert bool(torch.equal(torch.sort(copies[-1][:, 1]).values, src[:, 1]))
        part = prof.get("partition", {"ms": float("nan"), "launches": 1})
        part_ms = part["ms"] / max(1, part["launches"])
        out[dt] = {"gkeys_per_s": n / (ms * 1e-3) / 1e9, "ms": ms,
                   "partition_frac": partition_bytes(16, st) / (part_ms * 1e-3) / 1e9 / peak,
                   "leaf_ms": prof.get("leaves", {"ms": float("nan")})["ms"] / max(1, part["launches"])}
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
    """16,384 arrays, sizes log-uniform in [16, 65536], uniform u32 / f32
    keys: one autotuned segmented sort replayed as a CUDA graph vs one plain
    sort launch set per array, issued from Python and, without that
    overhead, captured into one CUDA graph. Outputs are compared byte for
    byte."""
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
        # the same per-array launches captured into one CUDA graph: the
        # baseline without Python and launch overhead
        eg = src.clone()
        pg, pstream = batch.capture_each(eg, off, dt, ws1)
        pg_ms = []
        for _ in range(max(1, reps // 2)):
            eg.copy_(src)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(pstream)
            with torch.cuda.stream(pstream):
                pg.replay()
            e1.record(pstream)
            torch.cuda.synchronize()
            pg_ms.append(e0.elapsed_time(e1))
        # bit patterns (f32 holds NaNs, which never compare equal as floats)
        same = bool(torch.equal(bits_view(graph_out, torch), bits_view(each, torch))) and \
            bool(torch.equal(bits_view(graph_out, torch), bits_view(eg, torch)))
        gm, pm, pgm = float(np.median(g_ms)), float(np.median(p_ms)), float(np.median(pg_ms))
        del pg, eg
        res[dt] = {"arrays": int(sizes.size), "keys": n, "graph_ms": gm, "per_array_ms": pm,
                   "per_array_graph_ms": pgm, "speedup_vs_per_array_graph": pgm / gm,
                   "graph_gkeys_per_s": n / (gm * 1e-3) / 1e9,
                   "per_array_gkeys_per_s": n / (pm * 1e-3) / 1e9, "speedup": pm / gm,
                   "identical_output": same, "tuned": tune["settings"],
                   "tuned_ms": tune["ms"], "default_ms": tune["default_ms"]}
        del b, src, each
        torch.cuda.empty_cache()
    return res


FIXED_RATE = 7500.0


def extra_served(vq, torch, num):
    """Poisson stream of `num` requests, sizes log-uniform in [1e3, 1e7],
    key type uniform over {i16, u32, f32, u64, kv64}, under a 40 GB budget:
    saturated capacity, then arrivals at 0.8 x capacity served with
    continuous batching (8 slots, one segmented sort per batch) and one at a
    time (plain). Every 50th request of the served run is compared, bit for
    bit, with the same keys sorted alone."""
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
    server.keep_ids = {r.rid for r in reqs[::50]}
    served = server.run(reqs)
    same = True
    for r in reqs[::50]:
        solo = vq.sort(r.source[r.offset:r.offset + r.n].clone(), r.dtype)
        same &= bool(torch.equal(bits_view(r.out, torch), bits_view(solo, torch)))
        r.out = None
    served["identical_output"] = same
    served["checked_requests"] = len(reqs[::50])
    # latency at a fixed arrival rate (7,500 requests/s), comparable across
    # builds whose saturated capacity differs
    fixed = server.run(serve.poisson_requests(num, FIXED_RATE, sources, seed=6))
    del server
    plain = serve.run_plain(serve.poisson_requests(num, rate, sources, seed=6), max_keys=hi)
    del sources
    torch.cuda.empty_cache()
    return {"requests": num, "rate_per_s": rate, "saturated": sat, "served": served, "plain": plain,
            "fixed_rate": dict(fixed, rate_per_s=FIXED_RATE),
            "throughput_ratio": served["gkeys_per_s"] / plain["gkeys_per_s"],
            "p99_ratio": plain["p99_ms"] / served["p99_ms"],
            "note": "plain is offered the same 0.8 x batched capacity, which exceeds its own, so its "
                    "latencies include queueing; throughput_ratio is the like-for-like figure"}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_2205_05982_gb300 as vq

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vq.load()
    if args.leaf_cutoff:
        vq.set_option("leaf_cutoff", args.leaf_cutoff)
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

    # every timed output is ordered and a permutation of the input
    if kb != 16:
        for c in copies[args.warmup:]:
            assert check_sorted_permutation(c, src, args.dtype, False, torch)
    del copies

    # rooflines: every kernel's algorithmic bytes per launch (2 x key bytes
    # per key it partitions or sorts) over its measured time per launch (CUDA
    # events on the launching stream); the slowest kernel is the dominant one
    peak, peak_kind = hbm_peak()

    def per_launch_ms(name):
        k = prof.get(name, {"ms": float("nan"), "launches": 1})
        return k["ms"] / max(1, k["launches"])

    part_ms = per_launch_ms("partition")
    part_bytes = partition_bytes(kb, st)
    achieved = part_bytes / (part_ms * 1e-3) / 1e9
    leaf_ms = per_launch_ms("leaves")   # the leaf phase, fork to join (its kernels overlap)
    sort_bytes = part_bytes + 2 * kb * args.n
    ideal = ideal_two_way(kb, args.n, vq.get_option("leaf_cutoff") or default_leaf_cutoff(kb, args.n))
    wl = f"{args.dtype}:{args.n}:{args.dist}"
    rooflines = {"partition": {
        "bound": "hbm", "kernel": "k_partition (persistent partition levels)", "achieved": achieved,
        "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
        "traffic": recorded_traffic(wl, KERNEL_SOURCES), "algorithmic_bytes_per_launch": part_bytes,
        "overhead_bytes_per_launch": partition_overhead_bytes(kb, st), "ms_per_launch": part_ms}}
    # The three leaf kernels run at once (block and warp leaves on side
    # streams forked from the sort's stream, mid leaves on it), so a leaf
    # kernel's time per launch includes time it shares the GPU with the
    # others; the leaf phase is read as a whole ("leaves", fork to join) as
    # well, and that is the figure compared with the partition.
    for name in ("leaf_block", "leaf_mid", "leaf_warp"):
        ms_l = per_launch_ms(name)
        byts = leaf_bytes(kb, st, name)
        got = byts / (ms_l * 1e-3) / 1e9 if ms_l > 0 else 0.0
        rooflines[name] = {"bound": "hbm", "kernel": f"k_{name}", "achieved": got, "peak": peak, "unit": "GB/s",
                           "frac": got / peak, "peak_source": peak_kind,
                           "traffic": recorded_traffic(f"{name}:{wl}", LEAF_SOURCES),
                           "algorithmic_bytes_per_launch": byts, "ms_per_launch": ms_l,
                           "concurrent_with": [k for k in ("leaf_block", "leaf_mid", "leaf_warp") if k != name]}
    # The leaf sorts are bound by the integer ALU pipe: the phase's ALU-pipe
    # warp instructions (ncu, recorded for the mid and block kernels; the
    # warp leaves, under 1 % of the keys, are not recorded) over the measured
    # ALU-pipe rate of the throughput probe; the HBM reading is beside it.
    leaf_total = sum(rooflines[k]["algorithmic_bytes_per_launch"] for k in ("leaf_block", "leaf_mid", "leaf_warp"))
    got = leaf_total / (leaf_ms * 1e-3) / 1e9 if leaf_ms > 0 else 0.0
    traffic = [rooflines[k]["traffic"] for k in ("leaf_block", "leaf_mid")]
    ipk = issue_peak()
    alus = [recorded_traffic(f"{k}:{wl}", LEAF_SOURCES, "alu_inst_per_launch") for k in ("leaf_block", "leaf_mid")]
    insts = [recorded_traffic(f"{k}:{wl}", LEAF_SOURCES, "inst_per_launch") for k in ("leaf_block", "leaf_mid")]
    alu = sum(alus) if all(alus) else None
    inst = sum(insts) if all(insts) else None
    keys = (st["leaf_keys_block"] + st["leaf_keys_mid"]) or 1
    alu_rate = alu / (leaf_ms * 1e-3) if alu and leaf_ms > 0 else None
    rooflines["leaves"] = {
        "bound": "alu", "kernel": "k_leaf_block + k_leaf_mid + k_leaf_warp (one phase, fork to join)",
        "achieved": alu_rate, "peak": ipk["warp_inst_per_s"], "unit": "ALU-pipe warp instructions/s",
        "frac": alu_rate / ipk["warp_inst_per_s"] if alu_rate else None,
        "peak_source": "measured (vqsort_probe_int_throughput)",
        "traffic": sum(traffic) if all(traffic) else None, "ms_per_launch": leaf_ms,
        "alu_inst_per_launch": alu, "inst_per_launch": inst,
        "thread_inst_per_key": inst * 32 / keys if inst else None,
        "comparisons_per_key": st["leaf_ce"] / max(1, st["leaf_keys"]),
        "hbm": {"achieved": got, "peak": peak, "unit": "GB/s", "frac": got / peak, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": leaf_total}}
    # the dominant step: the partition or the leaf phase, whichever is longer
    dominant = max(("partition", "leaves"), key=lambda k: rooflines[k]["ms_per_launch"]
                   if rooflines[k]["ms_per_launch"] == rooflines[k]["ms_per_launch"] else -1)
    kernels = {k: {"ms_per_launch": v["ms"] / max(1, v["launches"]), "launches": v["launches"]}
               for k, v in prof.items() if k != "leaves"}
    gpu_launches = sum(v["launches"] for k, v in prof.items() if k != "leaves")

    # end to end through the public host-buffer API: every step uploads its
    # own pinned array, sorts it and brings the keys back into it; steps
    # alternate between two streams (vqsort_sort_host_async), so one array
    # uploads while the other sorts and writes back over the other direction
    # of the host link. The single synchronous call is reported beside it.
    e2e_val = e2e_single = e2e_link = e2e_single_direct = e2e_trials = e2e_cpu = None
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
        # Inputs are staged into the pinned arrays before each trial, outside
        # the timed region, by a copy from the device-resident input (a DMA
        # write): on these machines pinned pages the CPU has just written are
        # slow for any GPU transfer, and more so the longer ago they were
        # written (plain copies of such arrays ran at 25-140 GB/s against
        # 340 GB/s otherwise), which is a property of the host, not of the
        # sort. The same loop on CPU-written arrays is reported beside it.
        src_bytes = src.reshape(-1).view(torch.uint8)

        def stage_gpu():
            for b in bufs:
                b.copy_(src_bytes, non_blocking=True)
            torch.cuda.synchronize()

        def stage_cpu():
            for v in views:
                v[...] = a

        def pipelined():
            t0 = time.perf_counter()
            for i in range(steps):
                vq.sort_host_async(views[i], args.dtype, stream=streams[i % 2])
            for st_ in streams:
                st_.synchronize()
            for st_ in streams:
                assert vq.last_device_status(None, st_) == 0
            return world * args.n * steps / (time.perf_counter() - t0) / 1e9

        trials, cpu_trials = [], []
        for _ in range(3):
            stage_gpu()
            trials.append(pipelined())
        if kb != 16:   # the last trial's outputs are ordered
            for v in views:
                o = torch.from_numpy(v.view({2: np.int16, 4: np.int32, 8: np.int64}[kb]))
                c = order_codes(o, args.dtype, torch)
                assert bool((c[1:] >= c[:-1]).all())
        for _ in range(2):
            stage_cpu()
            cpu_trials.append(pipelined())
        e2e_val = statistics.median(trials)
        # one synchronous call at a time (default copy-back, then the leaves'
        # direct stores into the pinned array), three calls each, median
        single, single_direct = [], []
        for direct, acc in ((0, single), (1, single_direct)):
            vq.set_option("host_direct", direct)
            for _ in range(3):
                bufs[0].copy_(src_bytes)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                vq.sort_host(views[0], args.dtype)
                acc.append(world * args.n / (time.perf_counter() - t0) / 1e9)
        vq.set_option("host_direct", 0)
        e2e_single = statistics.median(single)
        e2e_single_direct = statistics.median(single_direct)
        e2e_trials = [round(x, 3) for x in trials]
        e2e_cpu = [round(x, 3) for x in cpu_trials]
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
        # the first upload of each array right after the CPU rewrote them all
        stage_cpu()
        cpu_h2d = []
        for b in bufs:
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record()
            dev.copy_(b, non_blocking=True)
            c1.record()
            c1.synchronize()
            cpu_h2d.append(round(b.numel() / c0.elapsed_time(c1) / 1e6, 1))
        e2e_link = {"h2d_gbs": nbytes / h2d_med / 1e6, "d2h_gbs": nbytes / d2h_med / 1e6,
                    "copy_only_gkeys_per_s": args.n / ((h2d_med + d2h_med) * 1e-3) / 1e9,
                    "per_array_h2d_gbs": [round(nbytes / t / 1e6, 1) for t in h2d_ms],
                    "per_array_d2h_gbs": [round(nbytes / t / 1e6, 1) for t in d2h_ms],
                    "per_array_h2d_gbs_cpu_filled": cpu_h2d,
                    "how": "each pinned array of the timed loop up, then down, no sort (CUDA events, "
                           "best of 3 per array; the scalar rates are the medians); cpu_filled: one upload "
                           "of each array right after the CPU rewrote all of them"}
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
        "roofline": dict(rooflines[dominant], dominant_of=["leaves", "partition"]),
        "rooflines": rooflines,
        "issue_peak": ipk,
        "sort_roofline": {"how": "2 x key bytes x (keys of every partition level actually run + the leaf "
                                 "pass over all n keys) over the step time",
                          "bytes_per_step": sort_bytes,
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
                        "streams (upload, sort and copy-engine write-back of every step inside the timed "
                        "region); inputs staged into the pinned arrays by a device-to-host copy before each "
                        "trial; median of 3 trials",
                "trials": e2e_trials,
                "cpu_filled_trials": e2e_cpu,
                "cpu_filled_note": "the same loop right after the CPU rewrote every pinned array",
                "single_call": e2e_single, "single_call_path": "vqsort_sort_host (one array, waits; median of 3)",
                "single_call_leaf_stores": e2e_single_direct,
                "link": e2e_link},
        "clocks": clk,
    }
    if rank == 0:
        if not args.no_extras:
            vq.set_option("leaf_cutoff", 0)   # the extra workloads take the library's rule
            del src
            torch.cuda.empty_cache()
            line["c1"] = extra_c1(vq, torch)
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


def run_leaf_sizes(args):
    """Leaf microbenchmark: --n uniform keys of --dtype in CSR segments whose
    lengths are drawn uniformly from [LO, HI] (seeded); one segmented sort
    per step. Every segment is at most the leaf cutoff, so the sort is the
    leaf kernels alone (the partition kernel finds no work). Prints per-kernel
    times per launch and picoseconds per key."""
    import torch
    import paper_2205_05982_gb300 as vq
    vq.load()
    lo, hi = (int(x) for x in args.leaf_sizes.split(","))
    rng = np.random.default_rng(inputs.DEFAULT_SEED)
    sizes = rng.integers(lo, hi + 1, size=args.n // ((lo + hi) // 2) + 1)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    a = inputs.make(args.dtype, n, "uniform", specials=args.dtype in ("f32", "f64"))
    src = to_device_bits(a, args.dtype, torch)
    offd = torch.from_numpy(off.astype(np.int64)).cuda()
    ws = vq.alloc_workspace(args.dtype, n, sizes.size)
    copies = [src.clone() for _ in range(args.steps + args.warmup)]
    for i in range(args.warmup):
        vq.sort_segmented_ws_(copies[i], offd, ws, args.dtype)
    torch.cuda.synchronize()
    vq.profile_reset()
    vq.profile_enable(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for c in copies[args.warmup:]:
        vq.sort_segmented_ws_(c, offd, ws, args.dtype)
    e1.record()
    torch.cuda.synchronize()
    vq.profile_enable(False)
    prof = vq.profile_read()
    st = vq.stats(ws)
    assert st["device_status"] == 0 and st["keys_partitioned"] == 0, st
    ms = e0.elapsed_time(e1) / args.steps
    keys = {"leaf_warp": st["leaf_keys_warp"], "leaf_mid": st["leaf_keys_mid"], "leaf_block": st["leaf_keys_block"]}
    kern = {k: v["ms"] / max(1, v["launches"]) for k, v in prof.items()}
    print(json.dumps({"workload": f"leaf microbenchmark: {n} {args.dtype} keys in {sizes.size} segments of "
                                  f"{lo}..{hi} keys", "n_keys": n, "ms_per_step": ms,
                      "gkeys_per_s": n / (ms * 1e-3) / 1e9, "kernels_ms": kern, "leaf_keys": keys,
                      "ps_per_key": {k: kern[k] * 1e9 / keys[k] for k in keys if keys[k] and k in kern}}),
          flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.leaf_sizes:
        run_leaf_sizes(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
