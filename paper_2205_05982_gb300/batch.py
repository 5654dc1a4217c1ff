"""Batched sorting: thousands of independent arrays in one set of launches.

`SegmentedBatch` keeps a CSR batch of arrays resident on the device with its
workspace, sorts all segments with one `vqsort_sort_segmented_ws` call (the
same kernels as a plain sort, with every segment a root of the on-device
recursion) and can capture that call into a CUDA graph for replays. The
comparison baseline, `sort_each`, launches one plain sort per array.

`autotune` picks the partition tile size, the block-leaf keys per thread and
the leaf cutoff for a key type and a size distribution by timing candidate
settings on a sample batch; results are cached per (key type, size bucket)
in memory and, if `VQSORT_TUNING_CACHE` names a file, in that JSON file.
The output of a sort never depends on these settings, only its speed.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

import numpy as np

from . import CODE, KEY_BYTES, alloc_workspace, get_option, set_option, sort_segmented_ws_, sort_ws_

TUNABLES = ("tile_bytes", "leaf_cutoff", "leaf_threads")
DEFAULT = {"tile_bytes": 0, "leaf_cutoff": 0, "leaf_threads": 0}

_lock = threading.Lock()
_cache: dict = {}


def current_settings() -> dict:
    return {k: get_option(k) for k in TUNABLES}


def apply(settings: dict) -> None:
    for k in TUNABLES:
        set_option(k, int(settings.get(k, 0)))


class settings_scope:
    """Applies tuning settings for the duration of a `with` block."""

    def __init__(self, settings: dict | None):
        self.settings = settings
        self.saved = None

    def __enter__(self):
        if self.settings is not None:
            self.saved = current_settings()
            apply(self.settings)
        return self

    def __exit__(self, *exc):
        if self.saved is not None:
            apply(self.saved)
        return False


def candidates(dtype: str) -> list[dict]:
    """Valid (tile_bytes, leaf_cutoff, leaf_threads) combinations."""
    out = []
    kb = KEY_BYTES[dtype]
    cut_max = 4096 if kb == 16 else 16384
    for tile, cut, thr in itertools.product((16384, 32768, 65536), (2048, 4096, 8192, 16384), (0, 256, 512, 1024)):
        if cut > cut_max:
            continue
        if kb == 16 and thr:
            continue
        if thr and not (1 <= cut // thr <= 16):
            continue
        out.append({"tile_bytes": tile, "leaf_cutoff": cut, "leaf_threads": thr})
    return out


def size_bucket(n_total: int, num_segments: int) -> str:
    mean = n_total / max(1, num_segments)
    return f"n{int(np.log2(max(2, n_total)))}_m{int(np.log2(max(2, mean)))}"


class SegmentedBatch:
    """A resident CSR batch: `keys` (CUDA tensor) and `offsets` (num_segments+1)."""

    def __init__(self, keys, offsets, dtype: str, descending: bool = False, settings: dict | None = None):
        import torch
        self.keys = keys
        self.dtype = dtype
        self.descending = descending
        self.offsets = torch.as_tensor(np.asarray(offsets, dtype=np.int64)).to(keys.device)
        self.num_segments = self.offsets.numel() - 1
        self.n = keys.shape[0] if KEY_BYTES[dtype] == 16 else keys.numel()
        self.settings = settings
        with settings_scope(settings):
            self.ws = alloc_workspace(dtype, self.n, self.num_segments, device=keys.device)
        self.graph = None
        self.stream = None

    def sort(self, stream=None):
        with settings_scope(self.settings):
            sort_segmented_ws_(self.keys, self.offsets, self.ws, self.dtype, self.descending, stream)
        return self.keys

    def capture(self):
        """Records the segmented sort into a CUDA graph (one replay = one sort)."""
        import torch
        self.stream = torch.cuda.Stream(device=self.keys.device)
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            self.sort(self.stream)          # warm-up outside capture (lazy module loads)
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with settings_scope(self.settings):
            with torch.cuda.graph(self.graph, stream=self.stream):
                sort_segmented_ws_(self.keys, self.offsets, self.ws, self.dtype, self.descending,
                                   self.stream)
        return self.graph

    def replay(self):
        """Launches the captured graph on the batch's stream, ordered after
        the work already queued on the caller's current stream."""
        import torch
        if self.graph is None:
            self.capture()
        self.stream.wait_stream(torch.cuda.current_stream(self.keys.device))
        with torch.cuda.stream(self.stream):
            self.graph.replay()
        return self.keys


def sort_each(keys, offsets, dtype: str, ws=None, descending: bool = False, stream=None):
    """Baseline: one plain sort launch set per array (same kernels, one array
    at a time)."""
    off = np.asarray(offsets, dtype=np.int64)
    if ws is None:
        ws = alloc_workspace(dtype, int(np.diff(off).max(initial=1)), 1, device=keys.device)
    for s in range(off.size - 1):
        lo, hi = int(off[s]), int(off[s + 1])
        if hi - lo > 1:
            sort_ws_(keys[lo:hi], ws, dtype, descending, stream)
    return keys


def capture_each(keys, offsets, dtype: str, ws, descending: bool = False):
    """The per-array baseline captured into ONE CUDA graph: a replay launches
    one plain sort (its fixed kernel sequence) per array, back to back, with
    no host work between them. Returns (graph, stream)."""
    import torch
    stream = torch.cuda.Stream(device=keys.device)
    stream.wait_stream(torch.cuda.current_stream(keys.device))
    with torch.cuda.stream(stream):
        sort_each(keys, offsets, dtype, ws=ws, descending=descending, stream=stream)   # warm-up, uncaptured
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        sort_each(keys, offsets, dtype, ws=ws, descending=descending, stream=stream)
    return graph, stream


def _time_batch(batch: SegmentedBatch, reps: int) -> float:
    import torch
    src = batch.keys.clone()
    ms = []
    for _ in range(reps):
        batch.keys.copy_(src)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        batch.sort()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    batch.keys.copy_(src)
    return float(np.median(ms))


def _cache_file():
    return os.environ.get("VQSORT_TUNING_CACHE")


def _load_cache():
    path = _cache_file()
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                _cache.update(json.load(f))
        except (OSError, ValueError):
            pass


def _save_cache():
    path = _cache_file()
    if path:
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(_cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def autotune(keys, offsets, dtype: str, reps: int = 3, candidate_list=None, force: bool = False) -> dict:
    """Times every candidate setting on this batch (sorted from the same
    contents each time) and returns the fastest, with its time and the
    default's time. Cached per (key type, size bucket)."""
    n = keys.shape[0] if KEY_BYTES[dtype] == 16 else keys.numel()
    off = np.asarray(offsets, dtype=np.int64)
    key = f"{dtype}:{size_bucket(n, off.size - 1)}"
    with _lock:
        if not _cache:
            _load_cache()
        if key in _cache and not force:
            return _cache[key]
    results = []
    batch = SegmentedBatch(keys, off, dtype, settings=None)
    saved = current_settings()
    try:
        for cand in [DEFAULT] + list(candidate_list or candidates(dtype)):
            batch.settings = cand
            with settings_scope(cand):
                batch.ws = alloc_workspace(dtype, n, off.size - 1, device=keys.device)
            results.append((_time_batch(batch, reps), cand))
    finally:
        apply(saved)
    best_ms, best = min(results, key=lambda r: r[0])
    entry = {"settings": best, "ms": best_ms, "default_ms": results[0][0],
             "tried": len(results)}
    with _lock:
        _cache[key] = entry
        _save_cache()
    return entry


def tuned_settings(n_total: int, num_segments: int, dtype: str) -> dict | None:
    """The cached best settings for this shape, if autotune has seen it."""
    with _lock:
        if not _cache:
            _load_cache()
        e = _cache.get(f"{dtype}:{size_bucket(n_total, num_segments)}")
    return e["settings"] if e else None


__all__ = ["SegmentedBatch", "sort_each", "capture_each", "autotune", "tuned_settings", "candidates", "settings_scope",
           "CODE"]
