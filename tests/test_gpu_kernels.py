"""GPU parity of the two per-level kernels on their own: one Partition
(Sec. 2.1) and pivot sampling (Sec. 2.2), against the oracle."""
import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.gpu_util import to_dev, to_host
from tests.total_order import bit_rows

pytestmark = pytest.mark.gpu

ALL = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64", "u128", "kv64")


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("n", (1, 7, 1000, 16377, 100003, 2_000_001))
@pytest.mark.parametrize("ascending", (True, False))
def test_partition_matches_definition(vq, oracle_mod, dtype, n, ascending):
    """Left count exact; each side holds the oracle's side as a multiset."""
    a = inputs.kv_pairs(n, seed=n) if dtype == "kv64" else \
        inputs.make(dtype, n, "uniform", seed=n, specials=True)
    piv = a[n // 3]
    want, wl = oracle_mod.partition(a, piv, dtype, ascending)
    out, left = vq.partition(to_dev(a, dtype), piv, dtype, descending=not ascending)
    got = to_host(out, dtype, a)
    L = int(left.item())
    assert L == wl
    assert sorted(bit_rows(got[:L])) == sorted(bit_rows(want[:L]))
    assert sorted(bit_rows(got[L:])) == sorted(bit_rows(want[L:]))


@pytest.mark.parametrize("dtype", ALL)
@pytest.mark.parametrize("offset_keys", (0, 1, 3))
@pytest.mark.parametrize("ascending", (True, False))
def test_choose_pivot_matches_oracle(vq, oracle_mod, dtype, offset_keys, ascending):
    """The same SFC64 draws, 64-byte chunk geometry and rank-127 choice."""
    if dtype in ("u128", "kv64") and offset_keys % 1:
        pytest.skip()
    n = 50_000
    a = inputs.kv_pairs(n + 8, seed=3) if dtype == "kv64" else \
        inputs.make(dtype, n + 8, "uniform", seed=3, specials=True)
    t = to_dev(a, dtype)
    view = t[offset_keys:offset_keys + n]
    addr_mod64 = view.data_ptr() % 64
    seed = 0xABCDEF + offset_keys
    got = vq.choose_pivot(view, seed, dtype, descending=not ascending)
    want = oracle_mod.choose_pivot(a[offset_keys:offset_keys + n], dtype, addr_mod64, seed, ascending)
    g = got.cpu().numpy().view(a.dtype).reshape(-1)
    assert g.tobytes() == np.asarray(want).tobytes()


@pytest.mark.parametrize("dtype", ("f64", "u64", "f32", "u32", "i16", "u128"))
@pytest.mark.parametrize("lg", (16, 20, 24))
def test_partition_microbenchmark_sizes(vq, oracle_mod, dtype, lg):
    """The partition-only microbenchmark's workloads (one Partition of 2^lg
    uniform keys around the key at n/2; the paper times 2^24 doubles):
    left count exact, each side equal to the oracle's as a multiset."""
    n = 1 << lg
    a = inputs.make(dtype, n, "uniform", seed=lg)
    piv = a[n // 2]
    want, wl = oracle_mod.partition(a, piv, dtype, True)
    out, left = vq.partition(to_dev(a, dtype), piv, dtype)
    got = to_host(out, dtype, a)
    L = int(left.item())
    assert L == wl
    w = 16 if inputs.KEY_BYTES[dtype] == 16 else inputs.KEY_BYTES[dtype]
    view = {2: np.uint16, 4: np.uint32, 8: np.uint64, 16: np.uint64}[w]

    def rows(x):
        v = np.ascontiguousarray(x).view(view)
        if w == 16:
            v = v.reshape(-1, 2)
            return v[np.lexsort((v[:, 0], v[:, 1]))]
        return np.sort(v)
    assert np.array_equal(rows(got[:L]), rows(want[:L]))
    assert np.array_equal(rows(got[L:]), rows(want[L:]))
