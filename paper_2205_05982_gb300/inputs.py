"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no sorting arithmetic: it only draws key arrays, so the
CUDA path and the CPU oracle can be fed identical bytes. Every array is a
pure function of ``(seed, stream, index)`` through the counter-based
SplitMix64 generator (Steele, Lea, Flood 2014): the i-th word of a stream is
``mix(seed + stream * 2**32 + (i + 1) * 0x9E3779B97F4A7C15)`` with the
published SplitMix64 finaliser as ``mix``.

Workloads (the paper sorts uniform random keys, Tables sort1M/parsort100M):
  - ``uniform``: full bit range; float keys are uniform finite bit patterns
    (both signs, subnormals included), optionally with 0.1 % each of -0.0,
    +0.0, +inf, -inf and NaN (half 0x7FC00000-style, half sign-set) at
    seeded positions;
  - ``distinct16``: 16 seeded full-range values, index uniform in [0, 16);
  - ``equal``: one seeded value;
  - ``sorted`` / ``reverse``: the uniform array in ascending / descending
    numpy order;
  - ``organpipe``: a[i] = V(min(i, n-1-i)) with V monotone from [0, n/2)
    onto the type's range (the median-of-3 killer for first/mid/last pivots);
  - ``kv64``: uniform 64-bit key, value = original index, 10 % of keys
    overwritten by a copy of another seeded key;
  - segmented batches: sizes floor(exp(U(ln lo, ln hi))) in CSR offsets.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

DTYPES = ("i16", "u16", "i32", "u32", "f32", "i64", "u64", "f64", "u128", "kv64")
NUMPY_DTYPE = {
    "i16": np.int16, "u16": np.uint16, "i32": np.int32, "u32": np.uint32,
    "f32": np.float32, "i64": np.int64, "u64": np.uint64, "f64": np.float64,
    "u128": np.uint64, "kv64": np.uint64,
}
KEY_BYTES = {"i16": 2, "u16": 2, "i32": 4, "u32": 4, "f32": 4, "i64": 8, "u64": 8,
             "f64": 8, "u128": 16, "kv64": 16}
DISTRIBUTIONS = ("uniform", "distinct16", "equal", "sorted", "reverse", "organpipe")
DEFAULT_SEED = 0x22050598


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def words(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n uint64 words of stream ``stream``, indices [start, start + n)."""
    base = np.uint64((seed + (stream << 32)) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        return _mix(base + idx * GAMMA)


def _below(w: np.ndarray, k: int) -> np.ndarray:
    """Maps uint64 words to [0, k) by the high bits (k < 2**32)."""
    return ((w >> np.uint64(32)) * np.uint64(k)) >> np.uint64(32)


def _finite_float_bits(seed: int, stream: int, n: int, width: int) -> np.ndarray:
    """Uniform bit patterns whose exponent is not all-ones (finite floats)."""
    if width == 32:
        bits = (words(seed, stream, n) >> np.uint64(32)).astype(np.uint32)
        exp_mask, ut = np.uint32(0x7F800000), np.uint32
    else:
        bits = words(seed, stream, n)
        exp_mask, ut = np.uint64(0x7FF0000000000000), np.uint64
    redraw = 1
    bad = np.nonzero((bits & exp_mask) == exp_mask)[0]
    while bad.size:
        w = words(seed, stream + 1000 * redraw, bad.size, start=int(bad[0]))
        fresh = (w >> np.uint64(32)).astype(ut) if width == 32 else w
        bits[bad] = fresh
        bad = bad[(bits[bad] & exp_mask) == exp_mask]
        redraw += 1
    return bits


def uniform_bits(dtype: str, n: int, seed: int = DEFAULT_SEED, stream: int = 0) -> np.ndarray:
    """Uniform full-range keys as raw bit patterns viewed in the key dtype."""
    kb = KEY_BYTES[dtype]
    if dtype == "f32":
        return _finite_float_bits(seed, stream, n, 32).view(np.float32)
    if dtype == "f64":
        return _finite_float_bits(seed, stream, n, 64).view(np.float64)
    if kb == 16:
        out = np.empty((n, 2), dtype=np.uint64)
        out[:, 0] = words(seed, stream, n)
        out[:, 1] = words(seed, stream + 1, n)
        return out
    w = words(seed, stream, n) >> np.uint64(64 - 8 * kb)
    return w.astype({2: np.uint16, 4: np.uint32, 8: np.uint64}[kb]).view(NUMPY_DTYPE[dtype])


def inject_float_specials(a: np.ndarray, seed: int, stream: int = 7,
                          fraction: float = 0.001) -> np.ndarray:
    """Overwrites `fraction` of positions each with -0.0, +0.0, +inf, -inf and
    NaN (half positive quiet NaN, half sign-set quiet NaN), in place."""
    n = a.size
    k = int(n * fraction)
    if k == 0:
        return a
    if a.dtype == np.float32:
        ut = np.uint32
        specials = [0x80000000, 0x00000000, 0x7F800000, 0xFF800000]
        nans = (0x7FC00000, 0xFFC00000)
    else:
        ut = np.uint64
        specials = [0x8000000000000000, 0, 0x7FF0000000000000, 0xFFF0000000000000]
        nans = (0x7FF8000000000000, 0xFFF8000000000000)
    bits = a.view(ut)
    pos = words(seed, stream, 5 * k)
    idx = ((pos >> np.uint64(11)).astype(np.float64) * (n / 2.0 ** 53)).astype(np.int64)
    idx = np.minimum(idx, n - 1)
    for j, v in enumerate(specials):
        bits[idx[j * k:(j + 1) * k]] = ut(v)
    nan_idx = idx[4 * k:]
    bits[nan_idx[0::2]] = ut(nans[0])
    bits[nan_idx[1::2]] = ut(nans[1])
    return a


def organ_pipe(dtype: str, n: int) -> np.ndarray:
    """a[i] = V(min(i, n-1-i)), V monotone from [0, ceil(n/2)) onto the range."""
    half = max(1, (n + 1) // 2)
    k = np.minimum(np.arange(n, dtype=np.int64), n - 1 - np.arange(n, dtype=np.int64))
    frac = k.astype(np.float64) / max(1, half - 1)
    if dtype in ("f32", "f64"):
        ft = NUMPY_DTYPE[dtype]
        big = float(np.finfo(ft).max) / 2
        return (-big + frac * (2 * big)).astype(ft)
    kb = KEY_BYTES[dtype]
    if kb == 16:
        hi = (frac * float(2 ** 64 - 2 ** 12)).astype(np.uint64)
        out = np.empty((n, 2), dtype=np.uint64)
        out[:, 0] = k.astype(np.uint64)
        out[:, 1] = hi
        return out
    info = np.iinfo(NUMPY_DTYPE[dtype])
    if kb == 8:
        # stay exact in 64-bit integers: V(k) = min + k * floor(range / (half - 1))
        step = np.uint64(((1 << 64) - 1) // max(1, half - 1))
        with np.errstate(over="ignore"):
            v = k.astype(np.uint64) * step
            if dtype == "i64":
                v = v + np.uint64(1 << 63)   # shift [0, 2**64) onto [min, max]
        return v.view(NUMPY_DTYPE[dtype])
    span = float(int(info.max) - int(info.min))
    return (int(info.min) + np.floor(frac * span)).astype(np.int64).astype(NUMPY_DTYPE[dtype])


def make(dtype: str, n: int, dist: str = "uniform", seed: int = DEFAULT_SEED,
         specials: bool = False) -> np.ndarray:
    """One key array of a named distribution (see module docstring)."""
    if dist == "uniform":
        a = uniform_bits(dtype, n, seed, 0)
    elif dist == "distinct16":
        vals = uniform_bits(dtype, 16, seed, 11)
        a = vals[_below(words(seed, 12, n), 16)]
    elif dist == "equal":
        a = np.repeat(uniform_bits(dtype, 1, seed, 13), n, axis=0)
        if KEY_BYTES[dtype] != 16:
            a = a.reshape(n)
    elif dist in ("sorted", "reverse"):
        a = uniform_bits(dtype, n, seed, 0)
        if KEY_BYTES[dtype] == 16:
            order = np.lexsort((a[:, 0], a[:, 1]))
            a = a[order]
        else:
            a = np.sort(a)
        if dist == "reverse":
            a = a[::-1].copy()
    elif dist == "organpipe":
        a = organ_pipe(dtype, n)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    a = np.ascontiguousarray(a)
    if specials and dtype in ("f32", "f64") and dist == "uniform":
        inject_float_specials(a, seed)
    return a


def kv_pairs(n: int, seed: int = DEFAULT_SEED, dup_fraction: float = 0.10) -> np.ndarray:
    """(n, 2) uint64: column 0 a uniform key, column 1 the original index;
    `dup_fraction` of the keys are overwritten by a copy of another key."""
    out = np.empty((n, 2), dtype=np.uint64)
    out[:, 0] = words(seed, 21, n)
    out[:, 1] = np.arange(n, dtype=np.uint64)
    k = int(n * dup_fraction)
    if k and n > 1:
        dst = _below(words(seed, 22, k), n).astype(np.int64)
        src = _below(words(seed, 23, k), n).astype(np.int64)
        out[dst, 0] = out[src, 0].copy()
    return out


def segment_sizes(num_segments: int, lo: int, hi: int, seed: int = DEFAULT_SEED,
                  stream: int = 31) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))) sizes, int64."""
    w = words(seed, stream, num_segments)
    u = (w >> np.uint64(11)).astype(np.float64) / float(2 ** 53)
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


def offsets_from_sizes(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=off[1:])
    return off
