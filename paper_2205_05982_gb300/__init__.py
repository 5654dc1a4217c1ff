"""vqsort on GB300: Python binding of libvqsort.so.

Argument marshalling only: every step of a sort runs in the library's CUDA
kernels. PyTorch supplies device memory and streams. The entry points keep
the C names without the ``vqsort_`` prefix:

    sort_(t, dtype=None, descending=False)          in place, t a CUDA tensor
    sort(t, ...)                                    sorted copy
    sort_kv_(pairs, descending=False)               (n, 2) 64-bit {key, value}
    sort_segmented_(t, offsets, ...)                CSR segments, in place
    sort_ws_ / sort_segmented_ws_                   caller-owned workspace
    sort_host(array, dtype, descending=False)       numpy array, end to end
    partition(t, pivot, ...)  -> (out, left_count)  one Partition (Sec. 2.1)
    choose_pivot(t, seed, ...)                      pivot sampling (Sec. 2.2)

Key type names: i16 u16 i32 u32 f32 i64 u64 f64 u128 kv64. 16-byte keys are
(n, 2) int64/uint64 tensors: u128 rows are {low, high}, kv64 rows {key, value}.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

DTYPES = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64", "u128", "kv64")
CODE = {name: i for i, name in enumerate(DTYPES)}
KEY_BYTES = {"i16": 2, "u16": 2, "i32": 4, "u32": 4, "f32": 4, "i64": 8, "u64": 8,
             "f64": 8, "u128": 16, "kv64": 16}
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported device", 3: "out of memory",
          4: "CUDA error", 5: "timeout", 6: "internal capacity overflow"}
OPTIONS = {"depth_limit": 0, "leaf_cutoff": 1, "seed": 2, "spin_limit": 3, "test_stall": 4,
           "tile_bytes": 5, "leaf_threads": 6, "kway": 7, "host_direct": 8}


class VqError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} (status {status})")


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "keys_partitioned", "tiles", "segments", "leaves_warp", "leaves_block", "leaf_keys",
        "equal_ranges", "equal_keys", "degenerate", "fallback_ranges", "fallback_keys",
        "max_depth", "device_status", "keys_counted", "kway_ranges", "guard",
        "partition_blocks", "leaves_mid", "leaf_ce", "leaf_keys_warp", "leaf_keys_mid",
        "leaf_keys_block")]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libvqsort.so, building it first if it is missing or stale and
    nvcc is available. Raises if the library cannot be loaded: there is no
    fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.stale():
        try:
            _build.build()
        except Exception as e:  # noqa: BLE001 - reported below if the load fails
            if not os.path.exists(_build.LIB):
                raise ImportError(f"libvqsort.so is missing and could not be built: {e}") from e
    if not os.path.exists(_build.LIB):
        raise ImportError("libvqsort.so is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    vp, sz, i32, u64, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64
    sigs = {
        "vqsort_sort": ([i32, vp, sz, i32, vp], i32),
        "vqsort_sort_kv": ([vp, sz, i32, vp], i32),
        "vqsort_sort_kv_by_key": ([vp, sz, i32, vp], i32),
        "vqsort_sort_kv_by_key_ws": ([vp, sz, i32, vp, sz, vp], i32),
        "vqsort_sort_stable": ([i32, vp, sz, i32, vp, vp], i32),
        "vqsort_sort_host_async": ([i32, vp, sz, i32, vp], i32),
        "vqsort_sort_segmented": ([i32, vp, sz, vp, sz, i32, vp], i32),
        "vqsort_workspace_bytes": ([i32, sz, sz], sz),
        "vqsort_release_stream": ([vp], i32),
        "vqsort_sort_ws": ([i32, vp, sz, i32, vp, sz, vp], i32),
        "vqsort_sort_segmented_ws": ([i32, vp, sz, vp, sz, i32, vp, sz, vp], i32),
        "vqsort_sort_host": ([i32, vp, sz, i32], i32),
        "vqsort_partition": ([i32, vp, vp, sz, vp, i32, vp, vp], i32),
        "vqsort_choose_pivot": ([i32, vp, sz, u64, i32, vp, vp], i32),
        "vqsort_last_device_status": ([vp, vp], i32),
        "vqsort_device_status_async": ([vp, vp, vp], i32),
        "vqsort_get_stats": ([vp, vp, ctypes.POINTER(Stats)], i32),
        "vqsort_status_string": ([i32], ctypes.c_char_p),
        "vqsort_set_option": ([i32, i64], i32),
        "vqsort_get_option": ([i32], i64),
        "vqsort_merge_schedule": ([ctypes.c_uint, ctypes.c_uint, vp, sz, ctypes.POINTER(sz)], i32),
        "vqsort_profile_enable": ([i32], i32),
        "vqsort_profile_reset": ([], i32),
        "vqsort_profile_read": ([vp, vp, vp, sz, ctypes.POINTER(sz)], i32),
        "vqsort_probe_int_throughput": ([i32, ctypes.c_uint, ctypes.c_uint, vp, ctypes.POINTER(u64), vp], i32),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != 0:
        raise VqError(status, what)


# ----------------------------------------------------------------------------
# torch marshalling
# ----------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def infer_dtype(t) -> str:
    torch = _torch()
    m = {torch.int16: "i16", torch.int32: "i32", torch.float32: "f32", torch.int64: "i64",
         torch.float64: "f64"}
    for name, tn in (("u16", "uint16"), ("u32", "uint32"), ("u64", "uint64")):
        if hasattr(torch, tn):
            m[getattr(torch, tn)] = name
    if t.dtype not in m:
        raise TypeError(f"unsupported tensor dtype {t.dtype}")
    return m[t.dtype]


def _prep(t, dtype):
    if dtype is None:
        dtype = infer_dtype(t)
    if dtype not in CODE:
        raise ValueError(f"unknown key type {dtype!r}")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if KEY_BYTES[dtype] == 16:
        if t.dim() != 2 or t.shape[1] != 2 or t.element_size() != 8:
            raise ValueError("16-byte keys are (n, 2) tensors of 64-bit words")
        n = t.shape[0]
    else:
        if t.element_size() != KEY_BYTES[dtype]:
            raise ValueError(f"tensor element size does not match {dtype}")
        n = t.numel()
    return dtype, n


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def sort_(t, dtype: str | None = None, descending: bool = False, stream=None):
    """Sorts a CUDA tensor in place (library-owned workspace per stream)."""
    dtype, n = _prep(t, dtype)
    _check(load().vqsort_sort(CODE[dtype], ctypes.c_void_p(t.data_ptr()), n, int(not descending),
                              _stream(stream)), "vqsort_sort")
    return t


def sort(t, dtype: str | None = None, descending: bool = False, stream=None):
    return sort_(t.clone(), dtype, descending, stream)


def sort_kv_(pairs, descending: bool = False, stream=None):
    _, n = _prep(pairs, "kv64")
    _check(load().vqsort_sort_kv(ctypes.c_void_p(pairs.data_ptr()), n, int(not descending),
                                 _stream(stream)), "vqsort_sort_kv")
    return pairs


def sort_kv_by_key_(pairs, descending: bool = False, stream=None, ws=None):
    """Sorts (n, 2) 64-bit {key, value} rows in place by key alone (pairs
    with equal keys in an unspecified order)."""
    _, n = _prep(pairs, "kv64")
    if ws is None:
        _check(load().vqsort_sort_kv_by_key(ctypes.c_void_p(pairs.data_ptr()), n, int(not descending),
                                            _stream(stream)), "vqsort_sort_kv_by_key")
    else:
        p, nb = _ws_ptr(ws)
        _check(load().vqsort_sort_kv_by_key_ws(ctypes.c_void_p(pairs.data_ptr()), n, int(not descending), p, nb,
                                               _stream(stream)), "vqsort_sort_kv_by_key_ws")
    return pairs


def sort_stable_(t, dtype: str | None = None, descending: bool = False, stream=None):
    """Stable in-place sort (Sec. 5 row-id recipe); returns the int64 tensor
    of input positions of the output keys (equal keys keep input order)."""
    torch = _torch()
    dtype, n = _prep(t, dtype)
    rows = torch.empty(n, dtype=torch.int64, device=t.device)
    _check(load().vqsort_sort_stable(CODE[dtype], ctypes.c_void_p(t.data_ptr()), n, int(not descending),
                                     ctypes.c_void_p(rows.data_ptr()), _stream(stream)), "vqsort_sort_stable")
    return rows


def _offsets(offsets, device):
    torch = _torch()
    if not isinstance(offsets, torch.Tensor):
        offsets = torch.as_tensor(offsets, dtype=torch.int64)
    off = offsets.to(device=device, dtype=torch.int64).contiguous()
    return off


def sort_segmented_(t, offsets, dtype: str | None = None, descending: bool = False, stream=None):
    """Sorts segments [offsets[s], offsets[s+1]) of t independently, in place.
    offsets: 1-D integer tensor/array with num_segments + 1 entries."""
    dtype, n = _prep(t, dtype)
    off = _offsets(offsets, t.device)
    _check(load().vqsort_sort_segmented(CODE[dtype], ctypes.c_void_p(t.data_ptr()), n,
                                        ctypes.c_void_p(off.data_ptr()), off.numel() - 1,
                                        int(not descending), _stream(stream)),
           "vqsort_sort_segmented")
    return t


def workspace_bytes(dtype: str, n_total: int, num_segments: int = 1) -> int:
    return int(load().vqsort_workspace_bytes(CODE[dtype], n_total, num_segments))


def alloc_workspace(dtype: str, n_total: int, num_segments: int = 1, device=None):
    """A uint8 CUDA tensor large enough for a sort of this shape."""
    torch = _torch()
    return torch.empty(workspace_bytes(dtype, n_total, num_segments) + 256, dtype=torch.uint8,
                       device=device or "cuda")


def _ws_ptr(ws):
    p = ws.data_ptr()
    aligned = (p + 255) & ~255
    return ctypes.c_void_p(aligned), ws.numel() - (aligned - p)


def sort_ws_(t, ws, dtype: str | None = None, descending: bool = False, stream=None):
    dtype, n = _prep(t, dtype)
    p, nb = _ws_ptr(ws)
    _check(load().vqsort_sort_ws(CODE[dtype], ctypes.c_void_p(t.data_ptr()), n, int(not descending),
                                 p, nb, _stream(stream)), "vqsort_sort_ws")
    return t


def sort_segmented_ws_(t, offsets, ws, dtype: str | None = None, descending: bool = False,
                       stream=None):
    dtype, n = _prep(t, dtype)
    off = _offsets(offsets, t.device)
    p, nb = _ws_ptr(ws)
    _check(load().vqsort_sort_segmented_ws(CODE[dtype], ctypes.c_void_p(t.data_ptr()), n,
                                           ctypes.c_void_p(off.data_ptr()), off.numel() - 1,
                                           int(not descending), p, nb, _stream(stream)),
           "vqsort_sort_segmented_ws")
    return t


def sort_host(array, dtype: str, descending: bool = False):
    """End-to-end sort of a host numpy array in place (copies inside)."""
    import numpy as np
    a = array if array.flags["C_CONTIGUOUS"] else np.ascontiguousarray(array)
    n = a.shape[0] if KEY_BYTES[dtype] == 16 else a.size
    _check(load().vqsort_sort_host(CODE[dtype], ctypes.c_void_p(a.ctypes.data), n, int(not descending)),
           "vqsort_sort_host")
    if a is not array:
        array[...] = a
    return array


def sort_host_async(array, dtype: str, descending: bool = False, stream=None):
    """Enqueues the end-to-end sort of a C-contiguous host numpy array on
    `stream` (a torch.cuda.Stream or None) and returns at once; the array
    holds the sorted keys once the stream has passed the call. Keep the
    array alive and untouched until then."""
    if not array.flags["C_CONTIGUOUS"]:
        raise ValueError("sort_host_async needs a C-contiguous array")
    n = array.shape[0] if KEY_BYTES[dtype] == 16 else array.size
    _check(load().vqsort_sort_host_async(CODE[dtype], ctypes.c_void_p(array.ctypes.data), n, int(not descending),
                                         _stream(stream)), "vqsort_sort_host_async")
    return array


def partition(t, pivot, dtype: str | None = None, descending: bool = False, stream=None):
    """One Partition of t around `pivot` (a key: numpy scalar/row or bytes).
    Returns (out, left_count); out[:left_count] holds the keys <= pivot."""
    import numpy as np
    torch = _torch()
    dtype, n = _prep(t, dtype)
    out = torch.empty_like(t)
    left = torch.zeros(1, dtype=torch.int64, device=t.device)
    pb = pivot if isinstance(pivot, (bytes, bytearray)) else np.asarray(pivot).tobytes()
    if len(pb) != KEY_BYTES[dtype]:
        raise ValueError("pivot must be one key")
    buf = ctypes.create_string_buffer(pb, len(pb))
    _check(load().vqsort_partition(CODE[dtype], ctypes.c_void_p(t.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), n, buf, int(not descending),
                                   ctypes.c_void_p(left.data_ptr()), _stream(stream)),
           "vqsort_partition")
    return out, left


def choose_pivot(t, seed: int, dtype: str | None = None, descending: bool = False, stream=None):
    """Pivot by the sampling rule of Sec. 2.2 (as the sorter uses it)."""
    torch = _torch()
    dtype, n = _prep(t, dtype)
    out = torch.empty((1, 2) if KEY_BYTES[dtype] == 16 else 1, dtype=t.dtype, device=t.device)
    _check(load().vqsort_choose_pivot(CODE[dtype], ctypes.c_void_p(t.data_ptr()), n,
                                      seed & 0xFFFFFFFFFFFFFFFF, int(not descending),
                                      ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "vqsort_choose_pivot")
    return out


def _ws_arg(ws):
    if ws is None:
        return None
    return _ws_ptr(ws)[0]


def last_device_status(ws=None, stream=None) -> int:
    return int(load().vqsort_last_device_status(_ws_arg(ws), _stream(stream)))


def device_status_async(ws, host_word, stream=None):
    """Enqueues a copy of workspace `ws`'s device status word into
    `host_word` (a pinned 1-element int64 CPU tensor) on `stream`; read it
    once the stream has passed this point (0 = ok)."""
    _check(load().vqsort_device_status_async(_ws_arg(ws), ctypes.c_void_p(host_word.data_ptr()),
                                             _stream(stream)), "vqsort_device_status_async")


def stats(ws=None, stream=None) -> dict:
    st = Stats()
    _check(load().vqsort_get_stats(_ws_arg(ws), _stream(stream), ctypes.byref(st)), "vqsort_get_stats")
    return {f: int(getattr(st, f)) for f, _ in Stats._fields_}


def release_stream(stream=None):
    """Frees the library's workspace and side streams for `stream` (default:
    the current stream) after waiting for it."""
    _check(load().vqsort_release_stream(_stream(stream)), "vqsort_release_stream")


def status_string(status: int) -> str:
    return load().vqsort_status_string(status).decode()


def set_option(name: str, value: int):
    _check(load().vqsort_set_option(OPTIONS[name], int(value)), f"set_option({name})")


def get_option(name: str) -> int:
    return int(load().vqsort_get_option(OPTIONS[name]))


def merge_schedule(run_len: int, keys_per_thread: int = 1) -> list[list[tuple[int, int]]]:
    """The comparator pairs of one bitonic merge, grouped by step."""
    lib = load()
    n = ctypes.c_size_t(0)
    _check(lib.vqsort_merge_schedule(run_len, keys_per_thread, None, 0, ctypes.byref(n)),
           "vqsort_merge_schedule")
    buf = (ctypes.c_uint * (2 * n.value))()
    _check(lib.vqsort_merge_schedule(run_len, keys_per_thread, buf, n.value, ctypes.byref(n)),
           "vqsort_merge_schedule")
    pairs = [(buf[2 * i], buf[2 * i + 1]) for i in range(n.value)]
    per_step = run_len   # every step compares run_len pairs
    return [pairs[s:s + per_step] for s in range(0, len(pairs), per_step)]


def profile_enable(on: bool = True):
    _check(load().vqsort_profile_enable(int(on)), "vqsort_profile_enable")


def profile_reset():
    _check(load().vqsort_profile_reset(), "vqsort_profile_reset")


def profile_read() -> dict:
    lib = load()
    cnt = ctypes.c_size_t(0)
    _check(lib.vqsort_profile_read(None, None, None, 0, ctypes.byref(cnt)), "vqsort_profile_read")
    k = cnt.value
    names = (ctypes.c_char_p * k)()
    ms = (ctypes.c_double * k)()
    la = (ctypes.c_uint64 * k)()
    _check(lib.vqsort_profile_read(names, ms, la, k, ctypes.byref(cnt)), "vqsort_profile_read")
    return {names[i].decode(): {"ms": ms[i], "launches": int(la[i])} for i in range(k)}


def probe_int_throughput(kind: int = 0, iters: int = 4096, blocks: int | None = None, reps: int = 5) -> dict:
    """Times the integer throughput probe (kind 0: 32-bit min, kind 1: 64-bit
    compare-and-select min) with CUDA events; returns lane operations per
    second (best of `reps`) and what was run."""
    torch = _torch()
    if blocks is None:
        blocks = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 8
    sink = torch.empty(blocks * 256, dtype=torch.int32, device="cuda")
    ops = ctypes.c_uint64(0)
    s = torch.cuda.current_stream()
    lib = load()
    _check(lib.vqsort_probe_int_throughput(kind, blocks, iters, ctypes.c_void_p(sink.data_ptr()),
                                           ctypes.byref(ops), _stream(s)), "vqsort_probe_int_throughput")
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check(lib.vqsort_probe_int_throughput(kind, blocks, iters, ctypes.c_void_p(sink.data_ptr()),
                                               ctypes.byref(ops), _stream(s)), "vqsort_probe_int_throughput")
        e1.record(s)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    total = ops.value * blocks * 256
    return {"lane_ops_per_s": total / (best * 1e-3), "ms": best, "blocks": blocks, "threads": 256,
            "iters": iters, "ops_per_thread": ops.value}
