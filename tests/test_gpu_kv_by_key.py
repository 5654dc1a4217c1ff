"""Key-only order of 64-bit key / 64-bit value pairs (Sec. 2.4 pairs,
Sec. 5: Quicksort is not stable). Pairs with equal keys may come out in any
order, so the output is checked by invariants: the key column equals the
oracle's sort of the input keys byte for byte, the pairs are the input's
pairs (the same multiset of rows), and every value still sits beside its
key (inputs carry value = original index)."""
import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _pairs(n, dist, seed=1):
    a = inputs.kv_pairs(n, seed=seed)
    if dist == "equal":
        a[:, 0] = 0x0123456789ABCDEF
    elif dist == "distinct16":
        vals = inputs.uniform_bits("u64", 16, seed, 11)
        a[:, 0] = vals[inputs.words(seed, 12, n) % 16]
    elif dist == "edges":   # keys 0 and 2^64 - 1 (the leaves' sentinel values) among uniform ones
        a[::7, 0] = 0
        a[3::11, 0] = np.uint64(2**64 - 1)
    elif dist == "sorted":
        a[:, 0] = np.sort(a[:, 0])
    return a


def check_by_key(vq, oracle_mod, a, ascending):
    t = to_dev(a, "kv64")
    vq.sort_kv_by_key_(t, descending=not ascending)
    got = to_host(t, "kv64", a)
    assert vq.last_device_status() == 0
    assert vq.stats()["guard"] == 0
    want_keys = oracle_mod.sort(np.ascontiguousarray(a[:, 0]), "u64", True)
    if not ascending:
        want_keys = want_keys[::-1]
    assert np.array_equal(got[:, 0], want_keys), "key column differs from the oracle's sorted keys"
    # every value beside its own key (value = original index)
    assert np.array_equal(got[:, 0], a[got[:, 1].astype(np.int64), 0]), "a value left its key"
    # the same pairs: as rows, the output is a permutation of the input
    assert np.array_equal(np.sort(got[:, 1]), np.arange(len(a), dtype=np.uint64)), "pairs lost or duplicated"
    return got


@pytest.mark.parametrize("n", (0, 1, 2, 33, 513, 2049, 5003, 70001, 1_000_003))
@pytest.mark.parametrize("dist", ("uniform", "equal", "distinct16", "edges", "sorted"))
@pytest.mark.parametrize("ascending", (True, False))
def test_kv_by_key_invariants(vq, oracle_mod, n, dist, ascending):
    check_by_key(vq, oracle_mod, _pairs(n, dist, seed=n + 5), ascending)


def test_kv_by_key_c3_size(vq, oracle_mod):
    """2.5e7 pairs (uniform keys, 10 % duplicated, value = index)."""
    check_by_key(vq, oracle_mod, inputs.kv_pairs(25_000_000), True)


@pytest.mark.parametrize("limit", (0, 1, 3))
def test_kv_by_key_depth_bound_fallback(vq, oracle_mod, limit):
    old = vq.get_option("depth_limit")
    try:
        vq.set_option("depth_limit", limit)
        for dist in ("uniform", "edges", "distinct16"):
            check_by_key(vq, oracle_mod, _pairs(300_007, dist, seed=limit), True)
    finally:
        vq.set_option("depth_limit", old)


def test_kv_by_key_with_workspace(vq, oracle_mod):
    n = 200_003
    a = _pairs(n, "uniform", seed=9)
    ws = vq.alloc_workspace("kv64", n)
    for ascending in (True, False):
        t = to_dev(a, "kv64")
        vq.sort_kv_by_key_(t, descending=not ascending, ws=ws)
        got = to_host(t, "kv64", a)
        assert vq.last_device_status(ws) == 0
        want = oracle_mod.sort(np.ascontiguousarray(a[:, 0]), "u64", True)
        assert np.array_equal(got[:, 0], want if ascending else want[::-1])
        assert np.array_equal(got[:, 0], a[got[:, 1].astype(np.int64), 0])
