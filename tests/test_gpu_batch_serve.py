"""Batched and served forms: their outputs equal the oracle's, byte for byte,
whatever the tuning settings and whatever runs beside them."""
import numpy as np
import pytest

from paper_2205_05982_gb300 import inputs
from tests.gpu_util import same_bits, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ("u32", "f32", "u64"))
def test_segmented_graph_replay_and_per_array(vq, oracle_mod, dtype):
    from paper_2205_05982_gb300 import batch
    sizes = inputs.segment_sizes(600, 16, 65536, seed=2)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    a = inputs.make(dtype, n, "uniform", seed=2, specials=True)
    want = oracle_mod.sort_segmented(a, off, dtype, True)
    b = batch.SegmentedBatch(to_dev(a, dtype), off, dtype)
    b.capture()
    src = to_dev(a, dtype)
    for _ in range(2):
        b.keys.copy_(src)
        b.replay()
        b.stream.synchronize()
        assert same_bits(to_host(b.keys, dtype, a), want)
    each = to_dev(a, dtype)
    batch.sort_each(each, off, dtype)
    assert same_bits(to_host(each, dtype, a), want)


def test_autotune_picks_valid_settings(vq, oracle_mod):
    from paper_2205_05982_gb300 import batch
    sizes = inputs.segment_sizes(300, 16, 65536, seed=4)
    off = inputs.offsets_from_sizes(sizes)
    n = int(off[-1])
    a = inputs.make("u32", n, "uniform", seed=4)
    cands = batch.candidates("u32")[:6]
    before = batch.current_settings()
    res = batch.autotune(to_dev(a, "u32"), off, "u32", reps=1, candidate_list=cands, force=True)
    assert batch.current_settings() == before     # autotune puts the settings back
    assert res["settings"] in cands + [batch.DEFAULT]
    assert res["ms"] > 0 and res["tried"] == len(cands) + 1
    b = batch.SegmentedBatch(to_dev(a, "u32"), off, "u32", settings=res["settings"])
    b.sort()
    assert same_bits(to_host(b.keys, "u32", a), oracle_mod.sort_segmented(a, off, "u32", True))
    assert batch.current_settings() == before     # and so does a sort under tuned settings


def test_served_results_equal_solo_results(vq, oracle_mod):
    """Each request sorted in the mix (8 slots, overlapping on the GPU) equals
    the same request sorted alone (the oracle)."""
    import torch
    from paper_2205_05982_gb300 import serve
    hi = 200_000
    host = {dt: inputs.make(dt, hi, "uniform", seed=9, specials=dt == "f32") for dt in ("i16", "u32", "f32", "u64")}
    host["kv64"] = inputs.kv_pairs(hi, seed=9)
    sources = {dt: to_dev(v, dt) for dt, v in host.items()}
    reqs = serve.poisson_requests(80, 20000.0, sources, seed=3, lo=1000, hi=hi)
    server = serve.Server(slots=8, budget_bytes=8 * 10**9, max_keys=hi, keep_outputs=True)
    stats = server.run(reqs)
    assert stats["requests"] == 80 and stats["p99_ms"] >= stats["p50_ms"] > 0
    for r in reqs:
        src = host[r.dtype][r.offset:r.offset + r.n]
        want = oracle_mod.sort(src, r.dtype, True)
        got = to_host(r.out, r.dtype, src)
        assert same_bits(got, want), (r.rid, r.dtype, r.n)
    plain = serve.run_plain(reqs[:20], max_keys=hi, keep_outputs=True)
    assert plain["requests"] == 20
    for r in reqs[:20]:
        src = host[r.dtype][r.offset:r.offset + r.n]
        assert same_bits(to_host(r.out, r.dtype, src), oracle_mod.sort(src, r.dtype, True))
    torch.cuda.synchronize()
