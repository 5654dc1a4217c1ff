"""Seeded random configurations against the oracle: key type, size,
distribution, order and the library options that change the path (K-way
levels, tile window, leaf cutoff and threads) drawn together, so that
combinations no structured test names are exercised. Every result must equal
the oracle's byte for byte."""
import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.gpu_util import first_mismatch, same_bits, to_dev, to_host

pytestmark = pytest.mark.gpu

TYPES = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64", "u128", "kv64")
DISTS = ("uniform", "distinct16", "equal", "sorted", "reverse", "organpipe")
CASES = 480


def draw(case):
    r = np.random.default_rng(0x5EED0000 + case)
    dtype = TYPES[r.integers(len(TYPES))]
    n = int(np.exp(r.uniform(0, np.log(3_000_000))))
    dist = DISTS[r.integers(len(DISTS))]
    asc = bool(r.integers(2))
    opts = {"kway": int(r.integers(2)), "tile_bytes": int(r.choice([0, 16384, 32768, 65536])),
            "leaf_cutoff": int(r.choice([0, 1024, 2048, 4096, 8192, 16384])),
            "leaf_threads": int(r.choice([0, 256, 512, 1024]))}
    return dtype, n, dist, asc, opts


@pytest.mark.parametrize("case", range(CASES))
def test_fuzz_against_oracle(vq, oracle_mod, case):
    dtype, n, dist, asc, opts = draw(case)
    a = inputs.kv_pairs(n, seed=case) if (dtype == "kv64" and dist == "uniform") else \
        inputs.make(dtype, n, dist, seed=case, specials=dtype.startswith("f"))
    want = oracle_mod.sort(a, dtype, asc)
    for k, v in opts.items():
        vq.set_option(k, v)
    try:
        t = to_dev(a, dtype)
        vq.sort_(t, dtype, descending=not asc)
        got = to_host(t, dtype, a)
        st = vq.stats()
    finally:
        vq.set_option("kway", 1)
        for k in ("tile_bytes", "leaf_cutoff", "leaf_threads"):
            vq.set_option(k, 0)
    assert vq.last_device_status() == 0, (dtype, n, dist, asc, opts)
    assert st["guard"] == 0
    if not same_bits(got, want):
        i, cnt = first_mismatch(got, want)
        pytest.fail(f"{dtype} n={n} {dist} asc={asc} {opts}: {cnt} mismatches, first at {i}")


@pytest.mark.parametrize("case", range(80))
def test_fuzz_segmented_against_oracle(vq, oracle_mod, case):
    """Random CSR batches: 1..600 segments of log-uniform sizes (some empty,
    some one key, some large enough for K-way roots) under random options."""
    r = np.random.default_rng(0x5E60000 + case)
    dtype = TYPES[r.integers(len(TYPES))]
    nseg = int(r.integers(1, 600))
    hi = int(np.exp(r.uniform(np.log(16), np.log(400_000))))
    sizes = inputs.segment_sizes(nseg, 1, max(2, hi), seed=case)
    sizes[r.random(nseg) < 0.05] = 0
    sizes[r.random(nseg) < 0.05] = 1
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    dist = DISTS[r.integers(len(DISTS))]
    asc = bool(r.integers(2))
    a = inputs.kv_pairs(n, seed=case) if (dtype == "kv64" and dist == "uniform") else \
        inputs.make(dtype, n, dist, seed=case, specials=dtype.startswith("f"))
    want = oracle_mod.sort_segmented(a, off, dtype, asc)
    vq.set_option("kway", int(r.integers(2)))
    vq.set_option("leaf_cutoff", int(r.choice([0, 1024, 4096, 16384])))
    try:
        t = to_dev(a, dtype)
        vq.sort_segmented_(t, off.astype(np.int64), dtype, descending=not asc)
        got = to_host(t, dtype, a)
    finally:
        vq.set_option("kway", 1)
        vq.set_option("leaf_cutoff", 0)
    assert vq.last_device_status() == 0
    assert same_bits(got, want), (dtype, nseg, hi, dist, asc, first_mismatch(got, want))
