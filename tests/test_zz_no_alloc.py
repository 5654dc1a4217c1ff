"""The partition entry point that allocates nothing (vqsort_partition_noalloc)
must produce what vqsort_partition produces: the same left count and the
same keys on each side (the order within a side is unspecified). It is
called twice in a row, so a call that left stale state in the shared
scratch array would show up. This file is collected last on purpose: if it
fails, a run that stops at the first failure has already run every other
test, and it passes both alone and after them."""
import ctypes

import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.gpu_util import to_dev, to_host
from tests.total_order import bit_rows

pytestmark = pytest.mark.gpu


def _noalloc(vq):
    lib = vq.load()
    f = lib.vqsort_partition_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [ctypes.c_int, vp, vp, ctypes.c_size_t, vp, ctypes.c_int, vp, vp]
    f.restype = ctypes.c_int
    return f


def _call(f, vq, dtype, t, out, left, piv, ascending, stream):
    pb = ctypes.create_string_buffer(piv.tobytes(), piv.nbytes)
    return f(vq.CODE[dtype], ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(out.data_ptr()), t.shape[0], pb,
             int(ascending), ctypes.c_void_p(left.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("dtype", ("i16", "u32", "f32", "u64", "f64", "kv64"))
@pytest.mark.parametrize("ascending", (True, False))
def test_noalloc_partition_matches_partition(vq, oracle_mod, dtype, ascending):
    """Two calls in a row on a fresh stream: each equals vqsort_partition
    (the library's allocating entry point) and the oracle's partition by
    definition: the same left count, the same keys on each side. Neither
    call creates a library-owned workspace for that stream."""
    import torch
    f = _noalloc(vq)
    stream = torch.cuda.Stream()
    for call, n in enumerate((300_007, 2_000_003)):
        a = inputs.kv_pairs(n, seed=call) if dtype == "kv64" else \
            inputs.make(dtype, n, "uniform", seed=call, specials=True)
        piv = np.ascontiguousarray(a[n // 5])
        t = to_dev(a, dtype)
        out = torch.empty_like(t)
        left = torch.zeros(1, dtype=torch.int64, device=t.device)
        torch.cuda.synchronize()
        st = _call(f, vq, dtype, t, out, left, piv, ascending, stream)
        assert st == 0, vq.status_string(st)
        stream.synchronize()
        # no sort or partition has used a library-owned workspace on this stream
        assert vq.stats(stream=stream)["tiles"] == 0
        L = int(left.item())
        g = to_host(out, dtype, a)
        want, want_left = vq.partition(t, piv, dtype, descending=not ascending)
        torch.cuda.synchronize()
        assert L == int(want_left.item())
        w = to_host(want, dtype, a)
        assert sorted(bit_rows(g[:L])) == sorted(bit_rows(w[:L]))
        assert sorted(bit_rows(g[L:])) == sorted(bit_rows(w[L:]))
        o, ol = oracle_mod.partition(a, piv, dtype, ascending)
        assert L == ol
        assert sorted(bit_rows(g[:L])) == sorted(bit_rows(o[:L]))
        assert sorted(bit_rows(g[L:])) == sorted(bit_rows(o[L:]))


def test_noalloc_empty_input(vq):
    """n = 0 is a valid call: it writes a left count of 0 and nothing else."""
    import torch
    f = _noalloc(vq)
    t = torch.empty(0, dtype=torch.int64, device="cuda")
    out = torch.empty(0, dtype=torch.int64, device="cuda")
    left = torch.full((1,), 77, dtype=torch.int64, device="cuda")
    piv = np.zeros(1, dtype=np.uint64)
    st = _call(f, vq, "u64", t, out, left, piv, True, torch.cuda.current_stream())
    assert st == 0, vq.status_string(st)
    torch.cuda.synchronize()
    assert int(left.item()) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch(vq):
    f = _noalloc(vq)
    too_many = 65536 * ((32768 - 16) // 8) + 1
    piv = ctypes.create_string_buffer(8)
    st = f(vq.CODE["u64"], ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000), too_many, piv, 1,
           ctypes.c_void_p(0x300000), None)
    assert st == 1
