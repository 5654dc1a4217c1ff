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


@pytest.mark.parametrize("dtype", ("i16", "u32", "f32", "u64", "f64", "kv64"))
def test_noalloc_partition_matches_partition(vq, dtype):
    import torch
    f = _noalloc(vq)
    for call, n in enumerate((300_007, 2_000_003)):
        a = inputs.kv_pairs(n, seed=call) if dtype == "kv64" else \
            inputs.make(dtype, n, "uniform", seed=call, specials=True)
        piv = np.ascontiguousarray(a[n // 5])
        t = to_dev(a, dtype)
        want, want_left = vq.partition(t, piv, dtype)
        out = torch.empty_like(t)
        left = torch.zeros(1, dtype=torch.int64, device=t.device)
        pb = ctypes.create_string_buffer(piv.tobytes(), piv.nbytes)
        st = f(vq.CODE[dtype], ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(out.data_ptr()), n, pb, 1,
               ctypes.c_void_p(left.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, vq.status_string(st)
        torch.cuda.synchronize()
        L = int(left.item())
        assert L == int(want_left.item())
        g = to_host(out, dtype, a)
        w = to_host(want, dtype, a)
        assert sorted(bit_rows(g[:L])) == sorted(bit_rows(w[:L]))
        assert sorted(bit_rows(g[L:])) == sorted(bit_rows(w[L:]))


def test_noalloc_rejects_sizes_beyond_its_scratch(vq):
    f = _noalloc(vq)
    too_many = 65536 * ((32768 - 16) // 8) + 1
    piv = ctypes.create_string_buffer(8)
    st = f(vq.CODE["u64"], ctypes.c_void_p(0x100000), ctypes.c_void_p(0x200000), too_many, piv, 1,
           ctypes.c_void_p(0x300000), None)
    assert st == 1
