"""Helpers for GPU tests: numpy <-> CUDA tensors with exact bit patterns."""
import numpy as np

KEY_BYTES = {"i16": 2, "u16": 2, "i32": 4, "u32": 4, "f32": 4, "i64": 8, "u64": 8,
             "f64": 8, "u128": 16, "kv64": 16}
_SIGNED_VIEW = {2: np.int16, 4: np.int32, 8: np.int64}


def to_dev(a: np.ndarray, dtype: str):
    """Copies a key array to the GPU bit for bit. Unsigned keys travel as
    signed views of the same width (the library is told the key type)."""
    import torch
    kb = KEY_BYTES[dtype]
    if kb == 16:
        host = np.ascontiguousarray(a).view(np.int64).reshape(-1, 2)
    elif dtype in ("f32", "f64"):
        host = np.ascontiguousarray(a)
    else:
        host = np.ascontiguousarray(a).view(_SIGNED_VIEW[kb])
    return torch.from_numpy(host.copy()).cuda()


def to_host(t, dtype: str, like: np.ndarray) -> np.ndarray:
    h = t.cpu().numpy()
    return np.ascontiguousarray(h).view(like.dtype).reshape(like.shape)


def same_bits(x: np.ndarray, y: np.ndarray) -> bool:
    return x.shape == y.shape and np.ascontiguousarray(x).tobytes() == np.ascontiguousarray(y).tobytes()


def first_mismatch(x: np.ndarray, y: np.ndarray):
    bx = np.ascontiguousarray(x).view(np.uint8).reshape(x.shape[0], -1)
    by = np.ascontiguousarray(y).view(np.uint8).reshape(y.shape[0], -1)
    bad = np.nonzero((bx != by).any(axis=1))[0]
    return int(bad[0]) if bad.size else None, int(bad.size)
