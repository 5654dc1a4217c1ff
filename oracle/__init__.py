"""CPU oracle for the vqsort hot path -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It wraps ``oracle.cpp`` (plain scalar
C++, compiled with the host compiler) through ctypes and numpy. It shares no
code with the CUDA library in ``paper_2205_05982_gb300``.

Key types are named by strings: ``i16 u16 i32 u32 f32 i64 u64 f64 u128 kv64``.
Arrays of ``u128`` and ``kv64`` keys are numpy ``uint64`` arrays of shape
``(n, 2)``: for ``u128`` column 0 is the low word and column 1 the high word;
for ``kv64`` column 0 is the key and column 1 the value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

DTYPES = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64", "u128", "kv64")
_CODE = {name: i for i, name in enumerate(DTYPES)}
NUMPY_DTYPE = {
    "i16": np.int16, "u16": np.uint16, "i32": np.int32, "u32": np.uint32,
    "f32": np.float32, "i64": np.int64, "u64": np.uint64, "f64": np.float64,
    "u128": np.uint64, "kv64": np.uint64,
}
KEY_BYTES = {"i16": 2, "u16": 2, "i32": 4, "u32": 4, "f32": 4, "i64": 8, "u64": 8,
             "f64": 8, "u128": 16, "kv64": 16}


class Stats(ctypes.Structure):
    """Counters filled by one oracle sort."""
    _fields_ = [("heapsort_calls", ctypes.c_uint64), ("max_depth", ctypes.c_uint64),
                ("partitions", ctypes.c_uint64), ("degenerate", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (seconds)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, sz, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
            lib.oracle_encode.argtypes = [i32, vp, vp, sz, i32]
            lib.oracle_decode.argtypes = [i32, vp, vp, sz, i32]
            lib.oracle_sort.argtypes = [i32, vp, sz, i32, ctypes.c_int64, ctypes.POINTER(Stats)]
            lib.oracle_sort_segmented.argtypes = [i32, vp, vp, sz, i32]
            lib.oracle_partition.argtypes = [i32, vp, sz, vp, i32, vp, ctypes.POINTER(u64)]
            lib.oracle_sfc64.argtypes = [u64, vp, sz]
            lib.oracle_sfc64.restype = None
            lib.oracle_bounded.argtypes = [u64, u64]
            lib.oracle_bounded.restype = u64
            lib.oracle_median3.argtypes = [u64, u64, u64]
            lib.oracle_median3.restype = u64
            lib.oracle_choose_pivot.argtypes = [i32, vp, sz, u64, u64, i32, vp]
            _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise ValueError("oracle rejected its arguments")


def _keys(a: np.ndarray, dtype: str) -> np.ndarray:
    want = NUMPY_DTYPE[dtype]
    a = np.ascontiguousarray(a, dtype=want)
    if KEY_BYTES[dtype] == 16 and (a.ndim != 2 or a.shape[1] != 2):
        raise ValueError("128-bit keys are (n, 2) uint64 arrays")
    return a


def _n(a: np.ndarray, dtype: str) -> int:
    return a.shape[0] if KEY_BYTES[dtype] == 16 else a.size


def sort(keys: np.ndarray, dtype: str, ascending: bool = True, depth_limit: int = -1,
         with_stats: bool = False):
    """Returns a sorted copy of ``keys`` (Algorithm 1 with Heapsort fallback)."""
    out = _keys(keys, dtype).copy()
    st = Stats()
    _check(_load().oracle_sort(_CODE[dtype], out.ctypes.data, _n(out, dtype), int(ascending),
                               depth_limit, ctypes.byref(st)))
    if with_stats:
        return out, {f: getattr(st, f) for f, _ in Stats._fields_}
    return out


def sort_segmented(keys: np.ndarray, offsets: np.ndarray, dtype: str, ascending: bool = True):
    """Sorts each CSR segment ``[offsets[s], offsets[s+1])`` independently."""
    out = _keys(keys, dtype).copy()
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    _check(_load().oracle_sort_segmented(_CODE[dtype], out.ctypes.data, off.ctypes.data,
                                         off.size - 1, int(ascending)))
    return out


def encode(keys: np.ndarray, dtype: str, ascending: bool = True) -> np.ndarray:
    """Order-preserving codes: uint64 per key, or (n, 2) uint64 {low, high}."""
    a = _keys(keys, dtype)
    n = _n(a, dtype)
    out = np.zeros((n, 2) if KEY_BYTES[dtype] == 16 else n, dtype=np.uint64)
    _check(_load().oracle_encode(_CODE[dtype], a.ctypes.data, out.ctypes.data, n,
                                 int(ascending)))
    return out


def decode(codes: np.ndarray, dtype: str, ascending: bool = True) -> np.ndarray:
    c = np.ascontiguousarray(codes, dtype=np.uint64)
    n = c.shape[0]
    shape = (n, 2) if KEY_BYTES[dtype] == 16 else n
    out = np.zeros(shape, dtype=NUMPY_DTYPE[dtype])
    _check(_load().oracle_decode(_CODE[dtype], c.ctypes.data, out.ctypes.data, n,
                                 int(ascending)))
    return out


def sort_stable(keys: np.ndarray, dtype: str, ascending: bool = True):
    """Stable sort (Sec. 5: a unique row id appended below the key makes
    Quicksort stable). Returns (sorted keys, rows): rows[i] is the input
    position of output key i, and keys whose codes are equal keep their input
    order. By definition: order the rows by (code, row); numpy's lexsort is
    the library sort used as that step. 2-, 4- and 8-byte key types."""
    if KEY_BYTES[dtype] == 16:
        raise ValueError("stable sort covers 2-, 4- and 8-byte keys")
    a = _keys(keys, dtype)
    codes = encode(a, dtype, ascending)
    rows = np.lexsort((np.arange(codes.shape[0], dtype=np.uint64), codes)).astype(np.uint64)
    return a[rows], rows


def partition(keys: np.ndarray, pivot, dtype: str, ascending: bool = True):
    """Stable partition by definition: (out, left_count)."""
    a = _keys(keys, dtype)
    p = _keys(np.asarray(pivot).reshape((1, 2) if KEY_BYTES[dtype] == 16 else 1), dtype)
    out = np.empty_like(a)
    lc = ctypes.c_uint64(0)
    _check(_load().oracle_partition(_CODE[dtype], a.ctypes.data, _n(a, dtype), p.ctypes.data,
                                    int(ascending), out.ctypes.data, ctypes.byref(lc)))
    return out, int(lc.value)


def sfc64(seed: int, count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.uint64)
    _load().oracle_sfc64(seed, out.ctypes.data, count)
    return out


def bounded(draw: int, rng: int) -> int:
    return int(_load().oracle_bounded(draw, rng))


def median3(a: int, b: int, c: int) -> int:
    return int(_load().oracle_median3(a, b, c))


def choose_pivot(keys: np.ndarray, dtype: str, addr_mod64: int, seed: int,
                 ascending: bool = True):
    """Pivot by the GPU library's sampling rule; returns a key (numpy scalar or (2,) row)."""
    a = _keys(keys, dtype)
    out = np.zeros((1, 2) if KEY_BYTES[dtype] == 16 else 1, dtype=NUMPY_DTYPE[dtype])
    _check(_load().oracle_choose_pivot(_CODE[dtype], a.ctypes.data, _n(a, dtype), addr_mod64,
                                       seed, int(ascending), out.ctypes.data))
    return out[0]
