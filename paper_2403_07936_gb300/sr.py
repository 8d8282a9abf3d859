"""Weight blob packing for the SR prolongation generator (mg_load_prolong_weights).

Blob = 64-byte header {b"MGSRW001", u32 n_feat, u32 n_blocks, u32 n_params,
zero padding} followed by n_params little-endian float32 values in the order
in.w, in.b, in.a, per block (w1, b1, a, w2, b2), up.w, up.b, up.a, out.w, out.b.
Convolution weights are [out][in][3][3] (cross-correlation taps).
"""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"MGSRW001"
HEADER = 64


def layer_order(n_feat: int = 64, n_blocks: int = 8):
    """(name, shape) of every parameter in blob order."""
    out = [("in.w", (n_feat, 1, 3, 3)), ("in.b", (n_feat,)), ("in.a", (n_feat,))]
    for k in range(n_blocks):
        out += [(f"b{k}.w1", (n_feat, n_feat, 3, 3)), (f"b{k}.b1", (n_feat,)), (f"b{k}.a", (n_feat,)),
                (f"b{k}.w2", (n_feat, n_feat, 3, 3)), (f"b{k}.b2", (n_feat,))]
    out += [("up.w", (4 * n_feat, n_feat, 3, 3)), ("up.b", (4 * n_feat,)), ("up.a", (n_feat,)),
            ("out.w", (1, n_feat, 3, 3)), ("out.b", (1,))]
    return out


def pack_weights(weights: dict, n_feat: int = 64, n_blocks: int | None = None) -> bytes:
    """Serialise a {name: array} dict into the library's blob format."""
    if n_blocks is None:
        n_blocks = sum(1 for k in weights if k.endswith(".w1"))
    parts = []
    for name, shape in layer_order(n_feat, n_blocks):
        a = np.asarray(weights[name], dtype=np.float32)
        if a.shape != tuple(shape):
            raise ValueError(f"{name}: shape {a.shape} != {shape}")
        parts.append(a.ravel())
    flat = np.concatenate(parts).astype("<f4")
    header = MAGIC + struct.pack("<III", n_feat, n_blocks, flat.size)
    header += b"\0" * (HEADER - len(header))
    return header + flat.tobytes()


def unpack_weights(blob: bytes) -> dict:
    """Inverse of pack_weights (float32 arrays)."""
    if blob[:8] != MAGIC:
        raise ValueError("bad magic")
    n_feat, n_blocks, n = struct.unpack("<III", blob[8:20])
    flat = np.frombuffer(blob[HEADER:], dtype="<f4")
    if flat.size != n:
        raise ValueError("size mismatch")
    out, off = {}, 0
    for name, shape in layer_order(n_feat, n_blocks):
        k = int(np.prod(shape))
        out[name] = flat[off:off + k].reshape(shape).copy()
        off += k
    return out
