"""GPU parity: the CUDA sort through the C ABI must equal the CPU oracle
byte for byte (the sorted output is unique, so bit-exact is the bar)."""
import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.gpu_util import first_mismatch, same_bits, to_dev, to_host

pytestmark = pytest.mark.gpu

ALL = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64", "u128", "kv64")
# sizes around the warp-leaf limit (512), block-leaf cutoffs (4K/8K/16K),
# partition tile sizes (2047/4094/8188/16376 keys) and ragged tails
SIZES = (0, 1, 2, 33, 257, 513, 1025, 4097, 8193, 16385, 40001, 262147)


def make(dtype, n, dist, seed=1):
    if dtype == "kv64" and dist == "uniform":
        return inputs.kv_pairs(n, seed=seed)
    return inputs.make(dtype, n, dist, seed=seed, specials=True)


def check_sort(vq, oracle_mod, dtype, a, ascending):
    want = oracle_mod.sort(a, dtype, ascending)
    t = to_dev(a, dtype)
    vq.sort_(t, dtype, descending=not ascending)
    got = to_host(t, dtype, a)
    assert vq.last_device_status() == 0
    assert vq.stats()["guard"] == 0           # no range-bound guard fired
    if not same_bits(got, want):
        i, cnt = first_mismatch(got, want)
        pytest.fail(f"{dtype} n={len(a)} asc={ascending}: {cnt} mismatches, first at {i}")


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("n", SIZES)
def test_uniform_all_sizes(vq, oracle_mod, dtype, n):
    a = make(dtype, n, "uniform", seed=n + 3)
    check_sort(vq, oracle_mod, dtype, a, True)
    check_sort(vq, oracle_mod, dtype, a, False)


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("dist", ("distinct16", "equal", "sorted", "reverse", "organpipe"))
@pytest.mark.parametrize("n", (1000, 50001, 400009))
def test_distributions(vq, oracle_mod, dtype, dist, n):
    a = make(dtype, n, dist, seed=7)
    check_sort(vq, oracle_mod, dtype, a, True)
    check_sort(vq, oracle_mod, dtype, a, False)


@pytest.mark.parametrize("dtype", ("u64", "f32", "i16", "kv64"))
def test_one_million(vq, oracle_mod, dtype):
    a = make(dtype, 1_000_000, "uniform", seed=11)
    check_sort(vq, oracle_mod, dtype, a, True)


@pytest.mark.parametrize("dtype", ("u128", "kv64"))
def test_wide_keys_c3(vq, oracle_mod, dtype):
    """2.5e7 u128 keys / kv64 pairs with 10 % duplicated keys (pairing kept)."""
    n = 25_000_000
    a = inputs.kv_pairs(n) if dtype == "kv64" else inputs.make("u128", n)
    check_sort(vq, oracle_mod, dtype, a, True)
    if dtype == "kv64":
        t = to_dev(a, dtype)
        vq.sort_kv_(t)
        got = to_host(t, dtype, a)
        idx = got[:, 1].astype(np.int64)
        assert np.array_equal(got[:, 0], a[idx, 0])


@pytest.mark.parametrize("dtype", ("u32", "f32", "u64", "kv64"))
def test_segmented(vq, oracle_mod, dtype):
    sizes = inputs.segment_sizes(400, 16, 65536, seed=5)
    sizes[::37] = 0
    sizes[1::41] = 1
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    a = inputs.kv_pairs(n, seed=5) if dtype == "kv64" else inputs.make(dtype, n, "uniform", seed=5,
                                                                        specials=True)
    want = oracle_mod.sort_segmented(a, off, dtype, True)
    t = to_dev(a, dtype)
    vq.sort_segmented_(t, off.astype(np.int64), dtype)
    got = to_host(t, dtype, a)
    assert vq.last_device_status() == 0
    assert same_bits(got, want), first_mismatch(got, want)


def test_segmented_bad_offsets_reported(vq):
    import torch
    t = torch.zeros(100, dtype=torch.int32, device="cuda")
    vq.sort_segmented_(t, np.array([0, 50, 40, 100]), "u32")
    assert vq.last_device_status() == 1


def test_zero_one_principle_leaves(vq):
    """All 2**16 0/1 vectors of 16 keys as one segmented batch (warp
    networks), plus random 0/1 arrays that reach the block networks."""
    import torch
    x = np.arange(2 ** 16, dtype=np.uint32)
    bits = ((x[:, None] >> np.arange(16, dtype=np.uint32)[None, :]) & 1).astype(np.uint32).reshape(-1)
    off = np.arange(0, bits.size + 1, 16, dtype=np.int64)
    t = torch.from_numpy(bits.view(np.int32)).cuda()
    vq.sort_segmented_(t, off, "u32")
    got = t.cpu().numpy().view(np.uint32).reshape(-1, 16)
    assert (np.diff(got.astype(np.int64), axis=1) >= 0).all()
    assert np.array_equal(got.sum(axis=1), bits.reshape(-1, 16).sum(axis=1))
    rng = np.random.default_rng(0)
    for n in (600, 3000, 5000, 9000, 16000):
        b = rng.integers(0, 2, size=n).astype(np.uint64)
        tt = torch.from_numpy(b.view(np.int64)).cuda()
        vq.sort_(tt, "u64")
        g = tt.cpu().numpy().view(np.uint64)
        assert np.array_equal(g, np.sort(b))


def test_back_to_back_sorts_reuse_workspace(vq, oracle_mod):
    for n, seed in ((300_000, 1), (5_000, 2), (1_000_003, 3), (70_000, 4)):
        a = inputs.make("u32", n, "uniform", seed=seed)
        check_sort(vq, oracle_mod, "u32", a, True)


def test_explicit_workspace_and_graph_capture(vq, oracle_mod):
    """The workspace form allocates nothing, so a sort can be captured in a
    CUDA graph and replayed on new contents of the same buffer."""
    import torch
    n = 500_000
    a1 = inputs.make("u64", n, "uniform", seed=21)
    a2 = inputs.make("u64", n, "uniform", seed=22)
    t = to_dev(a1, "u64")
    ws = vq.alloc_workspace("u64", n)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        vq.sort_ws_(t, ws, "u64")
    s.synchronize()
    assert same_bits(to_host(t, "u64", a1), oracle_mod.sort(a1, "u64"))
    t.copy_(to_dev(a2, "u64"))
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vq.sort_ws_(t, ws, "u64")
    for src in (a1, a2):
        t.copy_(to_dev(src, "u64"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert same_bits(to_host(t, "u64", src), oracle_mod.sort(src, "u64"))


def test_graph_capture_on_a_fresh_stream(vq, oracle_mod):
    """A stream whose first sort is captured has no side streams yet: its leaf
    kernels are captured one after another on it, and the replay is exact."""
    import torch
    n = 700_001
    a = inputs.make("i64", n, "uniform", seed=31)
    t = to_dev(a, "i64")
    ws = vq.alloc_workspace("i64", n)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vq.sort_ws_(t, ws, "i64")
    for seed in (32, 33):
        b = inputs.make("i64", n, "uniform", seed=seed)
        t.copy_(to_dev(b, "i64"))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert same_bits(to_host(t, "i64", b), oracle_mod.sort(b, "i64"))


def test_sorts_interleaved_on_two_streams(vq, oracle_mod):
    """Sorts enqueued alternately on two streams, each with its own workspace
    and its own side streams for the leaf kernels, with no synchronisation
    between them, are each exact."""
    import torch
    n = 2_000_003
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    wss = [vq.alloc_workspace("u64", n) for _ in streams]
    arrays = [inputs.make("u64", n, "uniform", seed=40 + i) for i in range(6)]
    devs = [to_dev(x, "u64") for x in arrays]
    torch.cuda.synchronize()
    for i, t in enumerate(devs):
        with torch.cuda.stream(streams[i % 2]):
            vq.sort_ws_(t, wss[i % 2], "u64")
    torch.cuda.synchronize()
    for s, w in zip(streams, wss):
        assert vq.last_device_status(w, s) == 0
    for x, t in zip(arrays, devs):
        assert same_bits(to_host(t, "u64", x), oracle_mod.sort(x, "u64"))


def test_high_priority_stream(vq, oracle_mod):
    """A sort on a high-priority stream (its leaf kernels' side streams take
    that priority) is exact."""
    import torch
    s = torch.cuda.Stream(priority=-1)
    a = inputs.make("f32", 3_000_017, "uniform", seed=61)
    t = to_dev(a, "f32")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        vq.sort_(t, "f32", descending=True)
    s.synchronize()
    assert vq.last_device_status(None, s) == 0
    assert same_bits(to_host(t, "f32", a), oracle_mod.sort(a, "f32", False))
    vq.release_stream(s)


def test_release_stream(vq, oracle_mod):
    """Releasing a stream frees the library's workspace and side streams for
    it; the next sort on the stream creates them again and is exact."""
    import torch
    s = torch.cuda.Stream()
    for seed in (51, 52):
        a = inputs.make("u64", 1_000_003, "uniform", seed=seed)
        t = to_dev(a, "u64")
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            vq.sort_(t, "u64")
        s.synchronize()
        assert vq.last_device_status(None, s) == 0
        assert same_bits(to_host(t, "u64", a), oracle_mod.sort(a, "u64"))
        vq.release_stream(s)
    vq.release_stream(s)   # nothing held: a no-op


@pytest.mark.parametrize("kway", (0, 1))
@pytest.mark.parametrize("dtype", ("u32", "i64", "f64", "u128"))
@pytest.mark.parametrize("limit", (0, 1, 3))
def test_depth_bound_fallback(vq, oracle_mod, dtype, limit, kway):
    """Forcing the depth bound low sends ranges to the merge fallback; the
    result must not change. With K-way levels one level may already reach
    the leaves, so only the two-way run must reach the fallback."""
    vq.set_option("depth_limit", limit)
    vq.set_option("kway", kway)
    try:
        for dist in ("uniform", "organpipe", "distinct16"):
            n = 200_003
            a = make(dtype, n, dist, seed=9)
            check_sort(vq, oracle_mod, dtype, a, True)
            st = vq.stats()
            assert st["leaf_keys"] + st["equal_keys"] + st["fallback_keys"] == n
            assert st["max_depth"] <= limit
            if not kway or limit == 0:
                assert st["fallback_ranges"] >= 1
    finally:
        vq.set_option("depth_limit", -1)
        vq.set_option("kway", 1)


@pytest.mark.parametrize("cutoff", (1024, 4096, 16384))
def test_leaf_cutoff_option(vq, oracle_mod, cutoff):
    vq.set_option("leaf_cutoff", cutoff)
    try:
        for dtype in ("u16", "f32", "u64"):
            a = make(dtype, 300_001, "uniform", seed=cutoff)
            check_sort(vq, oracle_mod, dtype, a, False)
    finally:
        vq.set_option("leaf_cutoff", 0)


def test_bounded_wait_reports_timeout(vq, oracle_mod):
    """A tile whose count is never published: the next tile's bounded wait
    runs out, the sort reports VQ_ERR_TIMEOUT, and the next sort is fine."""
    import torch
    a = inputs.make("u32", 200_000, "uniform", seed=4)
    vq.set_option("spin_limit", 1 << 14)
    vq.set_option("test_stall", 1)
    try:
        t = to_dev(a, "u32")
        vq.sort_(t, "u32")
        assert vq.last_device_status() == 5
    finally:
        vq.set_option("test_stall", 0)
        vq.set_option("spin_limit", 1 << 22)
    torch.cuda.synchronize()
    check_sort(vq, oracle_mod, "u32", a, True)


def test_host_entry(vq, oracle_mod):
    a = inputs.make("f32", 2_000_003, "uniform", seed=31, specials=True)
    want = oracle_mod.sort(a, "f32", False)
    b = a.copy()
    vq.sort_host(b, "f32", descending=True)
    assert same_bits(b, want)


def pinned_like(a):
    """A page-locked host copy of `a` (numpy view of a pinned torch buffer)."""
    import torch
    buf = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True)
    v = buf.numpy().view(a.dtype).reshape(a.shape)
    v[...] = a
    return buf, v


@pytest.mark.parametrize("dtype,n,dist", [
    ("u64", 3_000_017, "uniform"), ("f32", 2_000_003, "uniform"), ("i16", 1_000_001, "distinct16"),
    ("u128", 500_009, "uniform"), ("kv64", 300_007, "uniform"), ("u32", 100_000, "equal"),
    ("u64", 1, "uniform"), ("f64", 5000, "uniform")])
@pytest.mark.parametrize("ascending", (True, False))
@pytest.mark.parametrize("direct", (0, 1))
def test_host_entry_pinned(vq, oracle_mod, dtype, n, dist, ascending, direct):
    """Pinned host buffers: copied back after the sort (default), or written
    by the leaf kernels directly (host_direct = 1)."""
    a = make(dtype, n, dist, seed=n % 101)
    want = oracle_mod.sort(a, dtype, ascending)
    keep, b = pinned_like(a)
    vq.set_option("host_direct", direct)
    try:
        vq.sort_host(b, dtype, descending=not ascending)
    finally:
        vq.set_option("host_direct", 0)
    assert same_bits(b, want)


@pytest.mark.parametrize("limit", (0, 2))
def test_host_entry_pinned_fallback(vq, oracle_mod, limit):
    """The depth-bound merge fallback writes the pinned buffer directly too."""
    a = make("u64", 200_003, "uniform", seed=3)
    want = oracle_mod.sort(a, "u64", True)
    vq.set_option("depth_limit", limit)
    try:
        keep, b = pinned_like(a)
        vq.sort_host(b, "u64")
    finally:
        vq.set_option("depth_limit", -1)
    assert same_bits(b, want)


def test_stats_are_consistent(vq):
    import torch
    n = 10_000_000
    a = inputs.make("u64", n, "uniform", seed=2)
    t = to_dev(a, "u64")
    vq.sort_(t, "u64")
    st = vq.stats()
    assert st["device_status"] == 0
    assert st["guard"] == 0
    assert st["leaf_keys"] + st["equal_keys"] + st["fallback_keys"] == n
    assert st["keys_partitioned"] >= n            # at least the root level
    assert st["max_depth"] <= 2 * 23 + 4
    torch.cuda.synchronize()


@pytest.mark.parametrize("kway", (0, 1))
@pytest.mark.parametrize("dtype", ("u16", "i32", "f32", "u64", "f64", "u128", "kv64"))
@pytest.mark.parametrize("dist", ("uniform", "distinct16", "equal", "sorted", "organpipe"))
def test_kway_levels_on_and_off(vq, oracle_mod, kway, dtype, dist):
    """Ranges of >= 2^18 keys are split 16 ways (counting + scatter pass) when
    the option is on; the output must not change."""
    vq.set_option("kway", kway)
    try:
        a = make(dtype, 1_500_007, dist, seed=13)
        check_sort(vq, oracle_mod, dtype, a, True)
        st = vq.stats()
        if kway and dist in ("uniform", "sorted", "organpipe"):
            assert st["kway_ranges"] >= 1
        if not kway:
            assert st["kway_ranges"] == 0
        check_sort(vq, oracle_mod, dtype, a, False)
    finally:
        vq.set_option("kway", 1)


@pytest.mark.parametrize("n", (30_000_000, 10_000_003))
def test_kway_mid_sizes_with_workspace(vq, oracle_mod, n):
    """Sizes whose second level is still K-way but whose third is two-way,
    through the caller-owned workspace form (as the benchmark calls it)."""
    a = inputs.make("u64", n, "uniform", seed=n % 97)
    want = oracle_mod.sort(a, "u64", True)
    ws = vq.alloc_workspace("u64", n)
    for _ in range(3):
        t = to_dev(a, "u64")
        vq.sort_ws_(t, ws, "u64")
        assert vq.last_device_status(ws) == 0, vq.stats(ws)
        assert vq.stats(ws)["guard"] == 0
        assert same_bits(to_host(t, "u64", a), want)


@pytest.mark.parametrize("dtype,n", [
    ("u64", 32_768), ("u64", 50_000), ("u64", 100_003), ("u64", 200_000), ("u64", 3_000_017),
    ("u32", 65_536), ("u32", 1_000_003), ("u16", 70_001), ("u16", 5_000_011),
    ("u128", 16_384), ("u128", 700_001), ("kv64", 400_009), ("f64", 20_000_003)])
def test_kway_bucket_counts(vq, oracle_mod, dtype, n):
    """Range sizes that give 16, 32, ..., 256 buckets (about a quarter of the
    4096-key leaf cutoff per bucket), and sizes whose buckets are split again,
    K ways or in two."""
    vq.set_option("leaf_cutoff", 4096)
    try:
        a = make(dtype, n, "uniform", seed=n % 1009)
        check_sort(vq, oracle_mod, dtype, a, True)
        st = vq.stats()
    finally:
        vq.set_option("leaf_cutoff", 0)
    assert st["kway_ranges"] >= 1
    assert st["keys_counted"] >= n            # the root range was counted
    assert st["leaf_keys"] + st["equal_keys"] + st["fallback_keys"] == n


@pytest.mark.parametrize("dtype,n,depth", [("u64", 1_000_000, 1), ("u32", 1_000_000, 1), ("f64", 500_000, 1)])
def test_short_arrays_default_cutoff(vq, oracle_mod, dtype, n, depth):
    """With no cutoff set, a short array takes the 16384-key cutoff: one
    K-way level of 256 buckets leaves leaves (a 4096-key cutoff would split
    most buckets again); a bucket that drew more than the cutoff from the
    short array's smaller splitter sample takes one two-way level."""
    a = make(dtype, n, "uniform", seed=5)
    check_sort(vq, oracle_mod, dtype, a, True)
    st = vq.stats()
    assert st["kway_ranges"] == 1
    assert st["max_depth"] <= depth + 1


@pytest.mark.parametrize("tile", (16384, 65536))
@pytest.mark.parametrize("dtype", ("u16", "u32", "u64", "u128"))
def test_kway_tile_windows(vq, oracle_mod, dtype, tile):
    """16 KiB tile windows (K-way tiles of half the default size, a smaller
    splitter sample) and 64 KiB windows (three blocks per SM)."""
    vq.set_option("tile_bytes", tile)
    try:
        a = make(dtype, 2_000_003, "uniform", seed=3)
        check_sort(vq, oracle_mod, dtype, a, True)
        assert vq.stats()["kway_ranges"] >= 1
        check_sort(vq, oracle_mod, dtype, a, False)
    finally:
        vq.set_option("tile_bytes", 0)


@pytest.mark.parametrize("dtype", ("u32", "u64", "kv64"))
def test_segmented_with_kway_roots(vq, oracle_mod, dtype):
    """CSR segments large enough to be split K ways next to small ones."""
    sizes = inputs.segment_sizes(60, 16, 2_000_000, seed=8)
    sizes[::7] = 0
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    a = inputs.kv_pairs(n, seed=8) if dtype == "kv64" else inputs.make(dtype, n, "uniform", seed=8)
    want = oracle_mod.sort_segmented(a, off, dtype, False)
    t = to_dev(a, dtype)
    vq.sort_segmented_(t, off.astype(np.int64), dtype, descending=True)
    got = to_host(t, dtype, a)
    assert vq.last_device_status() == 0
    st = vq.stats()
    assert st["guard"] == 0 and st["kway_ranges"] >= 1
    assert same_bits(got, want), first_mismatch(got, want)


@pytest.mark.parametrize("dtype", ("u64", "i16", "f32", "u128"))
def test_kway_equality_buckets_16_distinct(vq, oracle_mod, dtype):
    """16 distinct values: the splitters repeat, so the range is split in
    equality mode and every key lands in a bucket of one value, which is only
    copied: one K-way level, no two-way pass."""
    n = 2_000_003
    a = make(dtype, n, "distinct16", seed=21)
    check_sort(vq, oracle_mod, dtype, a, True)
    st = vq.stats()
    assert st["kway_ranges"] == 1
    assert st["equal_keys"] == n
    assert st["keys_partitioned"] == n


@pytest.mark.parametrize("dtype", ("u64", "u32", "f64"))
@pytest.mark.parametrize("ascending", (True, False))
def test_kway_equality_buckets_mixed(vq, oracle_mod, dtype, ascending):
    """Half the keys one repeated value, half uniform: the repeated value gets
    an equality bucket, the uniform keys around it are split further."""
    n = 3_000_017
    a = make(dtype, n, "uniform", seed=22)
    a[::2] = a[7]
    check_sort(vq, oracle_mod, dtype, a, ascending)
    st = vq.stats()
    assert st["equal_keys"] >= n // 2
    assert st["leaf_keys"] + st["equal_keys"] + st["fallback_keys"] == n


@pytest.mark.parametrize("threads", (256, 512, 1024))
@pytest.mark.parametrize("cutoff", (0, 4096, 16384))
def test_leaf_threads_with_any_cutoff(vq, oracle_mod, threads, cutoff):
    """A leaf thread count too small for the cutoff (16 keys per thread) is
    raised to cutoff/16; every combination sorts correctly."""
    vq.set_option("leaf_threads", threads)
    vq.set_option("leaf_cutoff", cutoff)
    try:
        for dtype in ("u64", "u32"):
            a = make(dtype, 400_003, "uniform", seed=threads + cutoff)
            check_sort(vq, oracle_mod, dtype, a, True)
    finally:
        vq.set_option("leaf_threads", 0)
        vq.set_option("leaf_cutoff", 0)


@pytest.mark.parametrize("ascending", (True, False))
def test_beyond_2_pow_31_keys(vq, ascending):
    """2^31 + 12345 u16 keys (4.3 GB), generated on the device: key indices,
    tile numbers and range cursors pass 2^31. The output must be sorted and
    hold the same multiset (its 65536-bin histogram); both are exact."""
    import torch
    n = (1 << 31) + 12345
    g = torch.Generator(device="cuda")
    g.manual_seed(1234)
    t = torch.randint(-32768, 32768, (n,), dtype=torch.int16, device="cuda", generator=g)
    want_hist = torch.bincount(t.view(torch.int16).to(torch.int32) + 32768, minlength=65536)
    vq.sort_(t, "u16", descending=not ascending)
    assert vq.last_device_status() == 0
    assert vq.stats()["guard"] == 0
    u = t.to(torch.int32) & 0xFFFF   # the u16 values
    step = 1 << 28
    for s0 in range(0, n - 1, step):   # adjacent pairs, in slices to bound memory
        a_, b_ = u[s0:min(n - 1, s0 + step)], u[s0 + 1:min(n, s0 + step + 1)]
        ok = bool((b_ >= a_).all()) if ascending else bool((b_ <= a_).all())
        assert ok, s0
    assert torch.equal(torch.bincount(t.to(torch.int32) + 32768, minlength=65536), want_hist)
    del t, u
    torch.cuda.empty_cache()


@pytest.mark.parametrize("direct", (0, 1))
def test_host_async_two_streams(vq, oracle_mod, direct):
    """Several host arrays, pinned and pageable, sorted on two streams at
    once: each ends up equal to the oracle's sort."""
    import torch
    vq.set_option("host_direct", direct)
    try:
        _host_async_two_streams(vq, oracle_mod, torch)
    finally:
        vq.set_option("host_direct", 0)


def _host_async_two_streams(vq, oracle_mod, torch):
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cases = [("u64", 3_000_017, True), ("f32", 2_000_003, False), ("i16", 1_000_001, True),
             ("u64", 2_500_001, False), ("kv64", 300_007, True)]
    keep, arrays, wants = [], [], []
    for i, (dtype, n, pinned) in enumerate(cases):
        a = make(dtype, n, "uniform", seed=40 + i)
        wants.append(oracle_mod.sort(a, dtype, i % 2 == 0))
        if pinned:
            buf, v = pinned_like(a)
            keep.append(buf)
        else:
            v = a.copy()
        arrays.append(v)
        vq.sort_host_async(v, dtype, descending=i % 2 == 1, stream=streams[i % 2])
    for s in streams:
        s.synchronize()
        assert vq.last_device_status(None, s) == 0
    for (dtype, n, _), v, w in zip(cases, arrays, wants):
        assert same_bits(v, w), dtype
