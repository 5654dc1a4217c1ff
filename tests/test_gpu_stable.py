"""GPU parity of the stable sort (Sec. 5 row-id recipe): the sorted keys and
the row permutation must equal the oracle's stable order byte for byte (the
permutation is unique: ties keep their input order)."""
import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.gpu_util import same_bits, to_dev, to_host

pytestmark = pytest.mark.gpu

TYPES = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64")


def check_stable(vq, oracle_mod, dtype, a, ascending):
    want_keys, want_rows = oracle_mod.sort_stable(a, dtype, ascending)
    t = to_dev(a, dtype)
    rows = vq.sort_stable_(t, dtype, descending=not ascending)
    assert vq.last_device_status() == 0
    assert vq.stats()["guard"] == 0
    got_rows = rows.cpu().numpy().astype(np.uint64)
    assert np.array_equal(got_rows, want_rows)
    assert same_bits(to_host(t, dtype, a), want_keys)


@pytest.mark.parametrize("dtype", TYPES)
@pytest.mark.parametrize("dist", ("uniform", "distinct16", "equal", "sorted", "reverse"))
@pytest.mark.parametrize("n", (1, 2, 1000, 100_003))
@pytest.mark.parametrize("ascending", (True, False))
def test_stable_matches_oracle(vq, oracle_mod, dtype, dist, n, ascending):
    a = inputs.make(dtype, n, dist, seed=n + 1, specials=dtype.startswith("f"))
    check_stable(vq, oracle_mod, dtype, a, ascending)


@pytest.mark.parametrize("dtype", ("u32", "i64", "f32"))
@pytest.mark.parametrize("dist", ("uniform", "distinct16"))
def test_stable_large(vq, oracle_mod, dtype, dist):
    """Sizes whose packed codes take the K-way levels."""
    a = inputs.make(dtype, 3_000_017, dist, seed=5)
    check_stable(vq, oracle_mod, dtype, a, dist == "uniform")


def test_stable_empty_and_unsupported(vq):
    import torch
    t = torch.empty(0, dtype=torch.int32, device="cuda")
    assert vq.sort_stable_(t, "u32").numel() == 0
    w = torch.zeros((8, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(vq.VqError) as e:
        vq.sort_stable_(w, "u128")
    assert e.value.status == 2   # VQ_ERR_UNSUPPORTED
