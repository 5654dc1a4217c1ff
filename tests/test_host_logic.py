"""Host-side logic that needs no GPU: request generation and statistics of
the serving loop, tuning candidates, and the multi-rank timing reduction of
bench.py on two gloo ranks."""
import os
import socket

import numpy as np
import pytest


class FakeSource:
    def __init__(self, n):
        self.shape = (n,)


def test_poisson_requests_shape():
    from paper_2205_05982_gb300 import serve
    src = {dt: FakeSource(10**7) for dt in ("i16", "u32", "f32", "u64", "kv64")}
    reqs = serve.poisson_requests(5000, 1000.0, src, seed=1)
    sizes = np.array([r.n for r in reqs])
    assert sizes.min() >= 1000 and sizes.max() <= 10**7
    # log-uniform: about half the requests below the geometric midpoint 1e5
    assert 0.45 < (sizes < 10**5).mean() < 0.55
    arr = np.array([r.arrival for r in reqs])
    assert arr[0] == 0 and (np.diff(arr) >= 0).all()
    assert abs(np.diff(arr).mean() - 1e-3) < 1e-4            # rate 1000/s
    kinds = {dt: sum(r.dtype == dt for r in reqs) for dt in src}
    assert min(kinds.values()) > 800
    assert all(0 <= r.offset <= 10**7 - r.n for r in reqs)


def test_summarize():
    from paper_2205_05982_gb300 import serve
    reqs = []
    for i in range(100):
        r = serve.Request(i, i * 0.001, "u32", 1000, None)
        r.done_ms = i + 2.0
        r.latency_ms = 2.0 + (i % 10)
        reqs.append(r)
    s = serve.summarize(reqs)
    assert s["requests"] == 100 and s["keys"] == 100_000
    assert s["p50_ms"] == pytest.approx(6.5) and s["p99_ms"] == pytest.approx(11.0)
    assert s["span_ms"] == pytest.approx(101.0 - 0.0)


def test_tuning_candidates_valid():
    from paper_2205_05982_gb300 import batch
    for dt in ("u16", "u32", "u64", "u128"):
        c = batch.candidates(dt)
        assert c
        for x in c:
            assert x["tile_bytes"] in (16384, 32768, 65536)
            if x["leaf_threads"]:
                assert 1 <= x["leaf_cutoff"] // x["leaf_threads"] <= 16
            if dt == "u128":
                assert x["leaf_cutoff"] <= 4096 and x["leaf_threads"] == 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(10.0 + rank, dist)
    q.put((rank, got))
    dist.destroy_process_group()


def test_bench_takes_max_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 11.0, 1: 11.0}


def test_ideal_two_way_roofline():
    import bench
    # 1e8 u64 keys, cutoff 8192: ceil(log2(12207.03)) = 14 levels + the leaf pass
    r = bench.ideal_two_way(8, 10**8, 8192)
    assert r["partition_levels"] == 14 and r["bytes"] == 2 * 10**8 * 8 * 15
    # exactly a power of two above the cutoff: 2^20 / 2^12 needs 8 halvings
    assert bench.ideal_two_way(4, 1 << 20, 4096)["partition_levels"] == 8
    # one leaf only
    assert bench.ideal_two_way(2, 4096, 4096) == {"bytes": 2 * 4096 * 2, "partition_levels": 0,
                                                   "leaf_cutoff": 4096}


def test_bench_default_cutoffs_match_library():
    """The bench's copy of the per-key-size default leaf cutoff agrees with
    the library's rule in launch.h."""
    import re
    import bench
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2205_05982_gb300", "csrc", "launch.h")).read()
    body = re.search(r"default_leaf_cutoff\(int kb\) \{\s*return ([^;]+);", src).group(1)
    expr = re.sub(r"(\d+)u\b", r"\1", body)

    def lib(kb):
        # the body is a chain of `kb == K ? V : ...` conditionals
        e = expr
        while "?" in e:
            m = re.match(r"\s*kb == (\d+) \? (\d+) : (.*)", e, re.S)
            if int(m.group(1)) == kb:
                return int(m.group(2))
            e = m.group(3)
        return int(e)

    for kb in (2, 4, 8, 16):
        assert bench.DEFAULT_LEAF_CUTOFF[kb] == lib(kb)

    # the size rule's bounds
    def const(name):
        return int(re.search(name + r" = 1ull << (\d+)", src).group(1))
    assert bench.LEAF_N_SMALL == {"wide": 1 << const("LEAF_N_SMALL_WIDE"), "narrow": 1 << const("LEAF_N_SMALL_NARROW")}
    assert bench.LEAF_N_MID == {"wide": 1 << const("LEAF_N_MID_WIDE"), "narrow": 1 << const("LEAF_N_MID_NARROW")}
    # 16384 for short arrays, 8192 for mid-size ones, the default for large
    # ones, segmented batches and 16-byte keys
    assert bench.default_leaf_cutoff(8, 10**6) == 16384
    assert bench.default_leaf_cutoff(8, 3 * 10**7) == 8192
    assert bench.default_leaf_cutoff(8, 10**8) == 4096
    assert bench.default_leaf_cutoff(4, 4 * 10**6) == 16384
    assert bench.default_leaf_cutoff(4, 6 * 10**7) == 4096
    assert bench.default_leaf_cutoff(8, 10**6, segments=16) == 4096
    assert bench.default_leaf_cutoff(16, 10**6) == 4096


def test_reference_sample_is_bounded():
    import bench
    assert bench.reference_sample_keys(10**8, 10, 3) == 10_000_000        # capped at 1e7
    assert bench.reference_sample_keys(10**8, 1000, 3) == int(bench.REFERENCE_SECONDS *
                                                              bench.ORACLE_KEYS_PER_S / 1003)
    assert bench.reference_sample_keys(10**8, 10**6, 0) == 100_000        # floor
    assert bench.reference_sample_keys(5000, 10, 3) == 5000               # never above n


def test_reference_arm_line():
    """bench.py --impl reference: one JSON line with the reference arm's
    keys, timing the oracle on the host for exactly --steps steps."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--n", "300000", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "GKeys/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GKeys/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
