"""Independent key order used to pin the oracle.

Written from definitions, not from the oracle's bit codec:
  - integers compare as mathematical integers (Python ``int``);
  - floats follow IEEE 754-2019 clause 5.10 ``totalOrder``: numerically
    ordered values compare numerically, ``-0 < +0``, a NaN with the sign bit
    set is below every non-NaN and a NaN without it above every non-NaN;
    among NaNs of one sign, a larger payload is further from zero;
  - u128 keys compare as the integer ``high * 2**64 + low``; kv64 pairs as the
    integer ``key * 2**64 + value``.
"""
from __future__ import annotations

import math
import struct

import numpy as np


def _float_parts(bits: int, width: int):
    if width == 32:
        x = struct.unpack("<f", struct.pack("<I", bits))[0]
        sign = bits >> 31
        payload = bits & 0x7FFFFF
    else:
        x = struct.unpack("<d", struct.pack("<Q", bits))[0]
        sign = bits >> 63
        payload = bits & 0xFFFFFFFFFFFFF
    return x, sign, payload


def float_key(bits: int, width: int):
    """A tuple whose Python ordering is totalOrder on the float with these bits."""
    x, sign, payload = _float_parts(bits, width)
    if math.isnan(x):
        # negative NaNs lowest (larger payload lower), positive NaNs highest
        return (0, -payload) if sign else (2, payload)
    if x == 0.0:
        return (1, 0.0, 1 if not sign else 0)
    return (1, x, 0)


def key_of(dtype: str):
    """Returns f(element) -> sortable Python object for one element."""
    if dtype in ("i16", "u16", "i32", "u32", "i64", "u64"):
        return lambda v: int(v)
    if dtype == "f32":
        return lambda v: float_key(int(np.float32(v).view(np.uint32)), 32)
    if dtype == "f64":
        return lambda v: float_key(int(np.float64(v).view(np.uint64)), 64)
    if dtype == "u128":
        return lambda row: (int(row[1]) << 64) | int(row[0])
    if dtype == "kv64":
        return lambda row: (int(row[0]) << 64) | int(row[1])
    raise ValueError(dtype)


def is_sorted(arr: np.ndarray, dtype: str, ascending: bool = True) -> bool:
    k = key_of(dtype)
    keys = [k(x) for x in arr]
    pairs = zip(keys, keys[1:])
    if ascending:
        return all(a <= b for a, b in pairs)
    return all(a >= b for a, b in pairs)


def bit_rows(arr: np.ndarray) -> list:
    """Elements as raw bytes, for bitwise comparisons and multisets."""
    a = np.ascontiguousarray(arr)
    if a.ndim == 2:
        return [bytes(r.tobytes()) for r in a]
    return [x.tobytes() for x in a]
