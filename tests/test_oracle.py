"""Pins for the CPU oracle, against things other than the oracle itself.

Each test names what fixes the expected result: brute force over all
permutations, a library routine (numpy sort, numpy's SFC64 bit generator),
the IEEE totalOrder definition (tests/total_order.py), closed forms, or
invariants that hold at any size.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.total_order import bit_rows, is_sorted, key_of

NARROW = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64")
ALL = NARROW + ("u128", "kv64")

# a few values per type, special floats included, used to build multisets
SPECIAL_BITS = {
    "f32": [0x80000000, 0x00000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00000,
            0x3F800000, 0xBF800000, 0x00000001, 0x80000001, 0x7F800001, 0xFFA00000],
    "f64": [0x8000000000000000, 0, 0x7FF0000000000000, 0xFFF0000000000000,
            0x7FF8000000000000, 0xFFF8000000000000, 0x3FF0000000000000,
            0xBFF0000000000000, 1, 0x8000000000000001],
}


def pool(dtype):
    """Small set of distinct keys covering the type's edges."""
    if dtype in ("f32", "f64"):
        ut = np.uint32 if dtype == "f32" else np.uint64
        ft = np.float32 if dtype == "f32" else np.float64
        return np.array(SPECIAL_BITS[dtype], dtype=ut).view(ft)
    if dtype in ("u128", "kv64"):
        v = [(0, 0), (1, 0), (0, 1), (2**64 - 1, 0), (0, 2**64 - 1), (5, 5), (2**63, 1)]
        return np.array(v, dtype=np.uint64)
    info = np.iinfo(inputs.NUMPY_DTYPE[dtype])
    return np.array([info.min, info.max, 0, 1, info.min + 1, info.max - 1, 7],
                    dtype=inputs.NUMPY_DTYPE[dtype])


def brute_force_sorted(arr, dtype, ascending):
    """All orderings of arr; keep those non-decreasing (or non-increasing)
    under the independent comparator; they must agree bit for bit."""
    k = key_of(dtype)
    rows = list(arr)
    keys = [k(r) for r in rows]
    found = None
    for perm in itertools.permutations(range(len(rows))):
        ks = [keys[i] for i in perm]
        ok = all((a <= b) if ascending else (a >= b) for a, b in zip(ks, ks[1:]))
        if ok:
            cand = [rows[i].tobytes() for i in perm]
            if found is None:
                found = cand
            else:
                assert cand == found, "two different sorted arrangements"
    return found


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("ascending", [True, False])
def test_bruteforce_all_multisets(oracle_mod, dtype, ascending):
    """Every multiset of size <= 5 over 3 keys of the pool, plus size-7 draws
    over 4 keys: the oracle equals the unique sorted permutation."""
    p = pool(dtype)
    rng = np.random.default_rng(1)
    cases = []
    for n in range(0, 6):
        for combo in itertools.product(range(3), repeat=n):
            cases.append(list(combo))
    for _ in range(40):
        cases.append(list(rng.integers(0, 4, size=7)))
    for _ in range(30):   # size 6 over the whole pool (more distinct specials)
        cases.append(list(rng.integers(0, len(p), size=6)))
    seen = 0
    for idx in cases:
        arr = p[np.array(idx, dtype=np.int64)] if idx else p[:0]
        got = oracle_mod.sort(arr, dtype, ascending)
        want = brute_force_sorted(arr, dtype, ascending) if len(idx) else []
        assert [r.tobytes() for r in got] == want, (dtype, idx)
        seen += 1
    assert seen > 300


@pytest.mark.parametrize("dtype", ["i16", "u16", "i32", "u32", "i64", "u64"])
@pytest.mark.parametrize("dist", inputs.DISTRIBUTIONS)
def test_integers_match_numpy_sort(oracle_mod, dtype, dist):
    """Library routine: numpy.sort orders integers exactly."""
    a = inputs.make(dtype, 20011, dist, seed=5)
    np.testing.assert_array_equal(oracle_mod.sort(a, dtype, True), np.sort(a))
    np.testing.assert_array_equal(oracle_mod.sort(a, dtype, False), np.sort(a)[::-1])


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_floats_match_numpy_and_totalorder(oracle_mod, dtype):
    """numpy.sort fixes the order of the non-NaN, non-zero keys; totalOrder
    fixes where -NaN, -0.0, +0.0 and +NaN go."""
    a = inputs.make(dtype, 50000, "uniform", seed=9, specials=True)
    got = oracle_mod.sort(a, dtype, True)
    ut = np.uint32 if dtype == "f32" else np.uint64
    sign = ut(1) << ut(8 * a.itemsize - 1)
    bits = got.view(ut)
    nan = np.isnan(got)
    neg_nan = nan & ((bits & sign) != 0)
    pos_nan = nan & ((bits & sign) == 0)
    n_neg, n_pos = int(neg_nan.sum()), int(pos_nan.sum())
    assert n_neg > 0 and n_pos > 0
    assert neg_nan[:n_neg].all() and pos_nan[len(got) - n_pos:].all()
    mid = got[n_neg:len(got) - n_pos]
    ref = np.sort(a[~np.isnan(a)])
    np.testing.assert_array_equal(mid, ref)                 # numeric order, zeros as one
    zeros = np.nonzero(mid == 0)[0]
    zb = mid[zeros].view(ut)
    assert ((zb & sign) != 0).sum() > 0 and ((zb & sign) == 0).sum() > 0
    nz = (zb & sign) != 0
    assert nz[: int(nz.sum())].all()                         # every -0.0 before every +0.0
    assert np.array_equal(np.sort(bits), np.sort(a.view(ut)))  # multiset of bit patterns
    desc = oracle_mod.sort(a, dtype, False)
    assert np.array_equal(desc.view(ut), got.view(ut)[::-1])


@pytest.mark.parametrize("dtype", ["u128", "kv64"])
@pytest.mark.parametrize("ascending", [True, False])
def test_wide_keys_match_lexsort(oracle_mod, dtype, ascending):
    """numpy.lexsort orders 128-bit numbers given (low, high) columns."""
    a = inputs.kv_pairs(30000, seed=3) if dtype == "kv64" else inputs.make("u128", 30000, seed=3)
    a[::7, 1 if dtype == "u128" else 0] = 5          # ties on the upper word
    hi, lo = (a[:, 1], a[:, 0]) if dtype == "u128" else (a[:, 0], a[:, 1])
    order = np.lexsort((lo, hi))
    want = a[order] if ascending else a[order][::-1]
    np.testing.assert_array_equal(oracle_mod.sort(a, dtype, ascending), want)


def test_kv_pairing_invariant(oracle_mod):
    """Every output pair occurred in the input: with value = original index,
    key == input[value].key."""
    a = inputs.kv_pairs(50000, seed=4)
    out = oracle_mod.sort(a, "kv64", True)
    idx = out[:, 1].astype(np.int64)
    np.testing.assert_array_equal(out[:, 0], a[idx, 0])
    assert np.array_equal(np.sort(idx), np.arange(a.shape[0]))


@pytest.mark.parametrize("dtype", ALL)
def test_heapsort_fallback_alone(oracle_mod, dtype):
    """depth_limit=0 runs Heapsort from the root: must equal the default path
    (and numpy for integers)."""
    a = inputs.make(dtype, 5000, "uniform", seed=2, specials=True)
    h, st = oracle_mod.sort(a, dtype, True, depth_limit=0, with_stats=True)
    assert st["heapsort_calls"] == 1 and st["partitions"] == 0
    q, st2 = oracle_mod.sort(a, dtype, True, with_stats=True)
    assert st2["heapsort_calls"] == 0
    assert bit_rows(h) == bit_rows(q)
    if dtype in NARROW and dtype not in ("f32", "f64"):
        np.testing.assert_array_equal(h, np.sort(a))


@pytest.mark.parametrize("dtype", ["i32", "u64", "i16"])
def test_organ_pipe_trips_depth_bound(oracle_mod, dtype):
    """Median-of-3 of first/mid/last on an organ pipe picks the minimum, so
    the 2*log2(n)+4 bound must hand the rest to Heapsort (Sec. 2.2)."""
    n = 40000
    a = inputs.make(dtype, n, "organpipe")
    out, st = oracle_mod.sort(a, dtype, True, with_stats=True)
    limit = 2 * (n.bit_length() - 1) + 4
    assert st["heapsort_calls"] >= 1
    assert st["max_depth"] <= limit
    np.testing.assert_array_equal(out, np.sort(a))


def test_all_equal_and_two_values_terminate(oracle_mod):
    """Degenerate-partition rule: all-equal ranges stop after one min/max
    scan; two distinct values make progress with the minimum as pivot."""
    a = np.full(100000, 7, dtype=np.uint32)
    out, st = oracle_mod.sort(a, "u32", True, with_stats=True)
    assert st["partitions"] == 1 and st["degenerate"] == 1
    np.testing.assert_array_equal(out, a)
    b = np.where(np.arange(100000) % 3 == 0, 9, 4).astype(np.uint32)[::-1].copy()
    out, st = oracle_mod.sort(b, "u32", True, with_stats=True)
    np.testing.assert_array_equal(out, np.sort(b))
    assert st["heapsort_calls"] == 0
    # the maximum repeated >= 1/3 of the time
    c = inputs.make("u32", 30000, "uniform", seed=8)
    c[::3] = np.iinfo(np.uint32).max
    np.testing.assert_array_equal(oracle_mod.sort(c, "u32", True), np.sort(c))


def _median3_network():
    """The modules of the paper's median-of-3 network (Sec. 2.2), read from
    tests/golden/median3_network.txt."""
    path = os.path.join(os.path.dirname(__file__), "golden", "median3_network.txt")
    with open(path) as f:
        nums = [int(x) for ln in f if not ln.startswith("#") for x in ln.split()]
    return list(zip(nums[0::2], nums[1::2]))


def test_median3_network_exhaustive(oracle_mod):
    """The paper's network, applied as compare-exchange modules, leaves the
    median of every 3-tuple (duplicates included) in slot 1, and the
    oracle's median3 returns that slot."""
    net = _median3_network()
    assert net == [(0, 2), (0, 1), (1, 2)]
    for t in list(itertools.product(range(3), repeat=3)) + list(itertools.permutations([0, 2**63, 2**64 - 1])):
        v = list(t)
        for i, j in net:
            if v[j] < v[i]:
                v[i], v[j] = v[j], v[i]
        assert v[1] == sorted(t)[1]
        assert oracle_mod.median3(*t) == v[1]


def _numpy_sfc64_stream(seed, count):
    """numpy's SFC64 bit generator with its state set to the published
    seeding (a = b = c = seed, counter = 1) and 12 outputs discarded."""
    bg = np.random.SFC64()
    st = bg.state
    st["state"]["state"] = np.array([seed, seed, seed, 1], dtype=np.uint64)
    st["has_uint32"] = 0
    bg.state = st
    return bg.random_raw(12 + count)[12:].astype(np.uint64)


@pytest.mark.parametrize("seed", [0, 1, 0x22050598, 2**64 - 1, 0x123456789ABCDEF])
def test_sfc64_matches_numpy(oracle_mod, seed):
    np.testing.assert_array_equal(oracle_mod.sfc64(seed, 1000), _numpy_sfc64_stream(seed, 1000))


def test_bounded_multiply_high(oracle_mod):
    """Closed form: floor(draw * range / 2**64), with Python big integers."""
    rng = np.random.default_rng(0)
    for _ in range(2000):
        d = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        r = int(rng.integers(1, 2**62))
        assert oracle_mod.bounded(d, r) == (d * r) >> 64
    assert oracle_mod.bounded(2**64 - 1, 10) == 9
    assert oracle_mod.bounded(0, 10) == 0


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("ascending", [True, False])
def test_partition_invariants(oracle_mod, dtype, ascending):
    """Left keys compare <= pivot, right keys > pivot under the independent
    order; both sides keep input order; the multiset is preserved."""
    a = inputs.make(dtype, 3001, "uniform", seed=6, specials=True)
    k = key_of(dtype)
    piv = a[1234]
    out, left = oracle_mod.partition(a, piv, dtype, ascending)
    kp = k(piv)
    if ascending:
        goes_left = [k(x) <= kp for x in a]
    else:
        goes_left = [k(x) >= kp for x in a]
    assert left == sum(goes_left)
    want = [x.tobytes() for x, g in zip(a, goes_left) if g] + \
           [x.tobytes() for x, g in zip(a, goes_left) if not g]
    assert bit_rows(out) == want


@pytest.mark.parametrize("dtype", ALL)
def test_encode_decode_round_trip_and_order(oracle_mod, dtype):
    """decode(encode(x)) == x bit for bit, and sorting the codes as unsigned
    integers agrees with the independent order (both directions)."""
    a = inputs.make(dtype, 4000, "uniform", seed=12, specials=True)
    if dtype in ("f32", "f64"):
        a = np.concatenate([a, pool(dtype)])
    for asc in (True, False):
        c = oracle_mod.encode(a, dtype, asc)
        back = oracle_mod.decode(c, dtype, asc)
        assert bit_rows(back) == bit_rows(a)
        if c.ndim == 2:
            order = np.lexsort((c[:, 0], c[:, 1]))
        else:
            order = np.argsort(c, kind="stable")
        assert is_sorted(a[order], dtype, asc)


@pytest.mark.parametrize("dtype", ["i16", "u16"])
def test_encode_exhaustive_16bit(oracle_mod, dtype):
    """All 2**16 patterns: codes are a bijection and order like integers."""
    a = np.arange(2**16, dtype=np.uint16).view(inputs.NUMPY_DTYPE[dtype])
    c = oracle_mod.encode(a, dtype, True)
    assert len(np.unique(c)) == 2**16
    np.testing.assert_array_equal(a[np.argsort(c)], np.sort(a))
    np.testing.assert_array_equal(oracle_mod.decode(c, dtype, True), a)


def test_encode_f32_totalorder_sampled(oracle_mod):
    """1e5 random f32 patterns (NaNs of every kind included) order by the
    totalOrder definition."""
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2**32, size=100000, dtype=np.uint64).astype(np.uint32)
    bits[:2000] |= np.uint32(0x7F800000)          # many NaN / inf patterns
    a = bits.view(np.float32)
    c = oracle_mod.encode(a, "f32", True)
    assert is_sorted(a[np.argsort(c, kind="stable")], "f32", True)


@pytest.mark.parametrize("dtype", ALL)
def test_segmented_equals_per_segment(oracle_mod, dtype):
    sizes = inputs.segment_sizes(40, 1, 300, seed=1)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    a = inputs.kv_pairs(n) if dtype == "kv64" else inputs.make(dtype, n, "uniform", seed=1)
    got = oracle_mod.sort_segmented(a, off, dtype, True)
    for s in range(40):
        lo, hi = int(off[s]), int(off[s + 1])
        assert bit_rows(got[lo:hi]) == bit_rows(oracle_mod.sort(a[lo:hi], dtype, True))
        assert is_sorted(got[lo:hi], dtype, True)


def _gather_sample(a, dtype, addr_mod64, seed):
    """The sample of the pivot rule built from library pieces: numpy's SFC64
    draws, Python big-integer multiply-high, plain index arithmetic."""
    kb = inputs.KEY_BYTES[dtype]
    kc = 64 // kb
    off = ((64 - addr_mod64) % 64) // kb
    n = a.shape[0]
    nc = (n - off) // kc
    draws = _numpy_sfc64_stream(seed, 256 // kc)
    rows = []
    for d in draws:
        first = off + ((int(d) * nc) >> 64) * kc
        rows.extend(a[first:first + kc])
    return rows


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("addr_mod64", [0, 16, 48])
@pytest.mark.parametrize("ascending", [True, False])
def test_choose_pivot_rule(oracle_mod, dtype, addr_mod64, ascending):
    """The pivot is the rank-127 element (in sort order) of the 256-key sample."""
    n = 5000
    a = inputs.kv_pairs(n, seed=7) if dtype == "kv64" else \
        inputs.make(dtype, n, "uniform", seed=7, specials=True)
    seed = 0xC0FFEE + addr_mod64
    rows = _gather_sample(a, dtype, addr_mod64, seed)
    assert len(rows) == 256
    k = key_of(dtype)
    rows.sort(key=k, reverse=not ascending)
    got = oracle_mod.choose_pivot(a, dtype, addr_mod64, seed, ascending)
    assert np.asarray(got).tobytes() == rows[127].tobytes()


@pytest.mark.parametrize("dtype", ("i16", "u32", "f32", "i64", "f64"))
@pytest.mark.parametrize("ascending", (True, False))
def test_sort_stable_matches_python_stable_sort(oracle_mod, dtype, ascending):
    """Pinned to Python's own stable sort (a merge sort, no code shared):
    rows in output order, keys by the total order, ties in input order."""
    rng = np.random.default_rng(11)
    a = inputs.make(dtype, 400, "distinct16", seed=5, specials=dtype.startswith("f"))
    a = a[rng.permutation(a.shape[0])]
    keys, rows = oracle_mod.sort_stable(a, dtype, ascending)
    codes = [int(c) for c in oracle_mod.encode(a, dtype, ascending)]
    want = sorted(range(len(codes)), key=lambda i: codes[i])   # stable by the language
    assert [int(r) for r in rows] == want
    assert np.ascontiguousarray(keys).tobytes() == np.ascontiguousarray(a[want]).tobytes()


def test_sort_stable_ties_keep_input_order(oracle_mod):
    """All-equal keys: the permutation is the identity, ascending or not."""
    a = np.full(17, 5, dtype=np.uint32)
    for asc in (True, False):
        _, rows = oracle_mod.sort_stable(a, "u32", asc)
        assert rows.tolist() == list(range(17))
