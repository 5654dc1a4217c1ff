"""Every one of the 2^32 f32 bit patterns through the sorter.

The 32-bit patterns are split by their top four bits into 16 chunks of 2^28;
each chunk is shuffled by an odd-multiplier permutation and sorted as f32
keys. Within one chunk every pattern has the same sign, so under IEEE 754
totalOrder (clause 5.10) a chunk sorts by its bit patterns: ascending for a
clear sign bit (larger patterns are larger magnitudes, then +inf, then NaNs
with growing payload) and descending for a set one (the mirror image). That
closed form is pinned against a comparator written from the IEEE definition
on windows that hold the zeros, the subnormals, the infinities and the NaN
boundaries (CPU test), and the GPU test checks every pattern of every chunk
in both orders against it. This file is collected after the other GPU test
files so that a run stopping at its first failure has run them already."""
import numpy as np
import pytest

from tests.total_order import float_key

CHUNK_BITS = 28
MULT = 0x5BD1E995   # odd: j -> j * MULT mod 2^k permutes [0, 2^k)


def chunk_sorted(h: int, lo: int, m: int, xp):
    """Ascending totalOrder of the m patterns (h << 28) | [lo, lo + m), as
    unsigned 32-bit values in an int64 array of module `xp` (numpy or torch
    on the device)."""
    base = (h << CHUNK_BITS) + lo
    k = xp.arange(m, dtype=xp.int64) if xp is np else xp.arange(m, dtype=xp.int64, device="cuda")
    return base + k if h < 8 else base + (m - 1) - k


def as_int32(u):
    """Unsigned 32-bit values in int64 -> the same bits as int32 values."""
    return u - ((u >> 31) << 32)


@pytest.mark.parametrize("h", range(16))
@pytest.mark.parametrize("lo", (0, 0x007FF800, 0x07FFF800, 0x0F7FF800, 0x0FFFF000))
def test_chunk_closed_form_is_total_order(h, lo):
    """The closed form equals Python's sort by the IEEE totalOrder key on
    4096-pattern windows: zeros and subnormals (lo = 0 in chunks 0 and 8),
    the smallest normals, mid exponents, the largest finite values with the
    infinities and the first NaNs (0x0F7FF800 in chunks 7 and 15), and the
    largest NaN payloads (0x0FFFF000)."""
    m = 4096
    pats = [(h << CHUNK_BITS) | (lo + i) for i in range(m)]
    want = sorted(pats, key=lambda b: float_key(b, 32))
    got = chunk_sorted(h, lo, m, np)
    assert [int(x) for x in got] == want


def test_shuffle_is_a_permutation():
    m = 1 << 16
    j = np.arange(m, dtype=np.int64)
    assert np.array_equal(np.sort((j * MULT + 12345) & (m - 1)), j)


@pytest.mark.gpu
@pytest.mark.parametrize("ascending", (True, False))
def test_every_f32_pattern(vq, ascending):
    import torch
    m = 1 << CHUNK_BITS
    j = torch.arange(m, dtype=torch.int64, device="cuda")
    perm = (j * MULT + 12345) & (m - 1)   # a permutation of [0, 2^28)
    del j
    for h in range(16):
        t = as_int32((h << CHUNK_BITS) | perm).to(torch.int32)
        vq.sort_(t.view(torch.float32), "f32", descending=not ascending)
        assert vq.last_device_status() == 0, h
        want = chunk_sorted(h, 0, m, torch)
        if not ascending:
            want = want.flip(0)
        assert torch.equal(t, as_int32(want).to(torch.int32)), h
        del t, want
    del perm
    torch.cuda.empty_cache()
