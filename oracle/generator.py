"""Plain FP64 CPU oracle of the super-resolution (SR) prolongation.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product library.

The paper replaces the multigrid prolongation by the generator of an SRGAN
(Sec. 2.3 and Fig. 1b, after Ledig et al.; Sec. 3.1; Appendix A, Algorithm 5).
The generator here is the one-channel, whole-grid variant:

    G = conv3x3(1 -> 64) + PReLU
        -> 8 x [ y = x + conv3x3(PReLU(conv3x3(x))) ]      (64 -> 64 each)
        -> conv3x3(64 -> 256) -> pixel-shuffle x2 -> PReLU
        -> conv3x3(64 -> 1)

All convolutions are 3x3 cross-correlations with bias and circular padding
(the error fields are periodic, so the windowing and stitching of Sec. 3.1
becomes plain periodic convolution over the whole grid).  PReLU has one slope
per channel.  Pixel-shuffle: out[c, 2y + dy, 2x + dx] = in[4c + 2dy + dx, y, x].

SR prolongation of a coarse error e_c (Algorithm 5, with a linear scale in
place of the symmetric-log normalisation of Algorithms 3-4):
    s = max |e_c| (s = 1 when e_c = 0),
    e_f = P_cubic e_c + s * G(e_c / s).

Optional bf16 emulation rounds (round-to-nearest-even) the weights of every
layer and the activations at the layer boundaries where the GPU path stores
bf16 tensors, so that the two can be compared tightly.
"""
from __future__ import annotations

import numpy as np

from .multigrid import prolong_cubic

N_FEAT = 64
N_BLOCKS = 8


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of the IEEE binary32 pattern; rounding adds
    0x7FFF plus the lowest kept bit before truncating.
    """
    f32 = np.asarray(a, dtype=np.float32)
    bits = f32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (rounded & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def weight_shapes(n_feat: int = N_FEAT, n_blocks: int = N_BLOCKS):
    """Ordered (name, shape) list of the generator's parameters."""
    shapes = [("in.w", (n_feat, 1, 3, 3)), ("in.b", (n_feat,)), ("in.a", (n_feat,))]
    for k in range(n_blocks):
        shapes += [(f"b{k}.w1", (n_feat, n_feat, 3, 3)), (f"b{k}.b1", (n_feat,)),
                   (f"b{k}.a", (n_feat,)),
                   (f"b{k}.w2", (n_feat, n_feat, 3, 3)), (f"b{k}.b2", (n_feat,))]
    shapes += [("up.w", (4 * n_feat, n_feat, 3, 3)), ("up.b", (4 * n_feat,)),
               ("up.a", (n_feat,)),
               ("out.w", (1, n_feat, 3, 3)), ("out.b", (1,))]
    return shapes


def shift2d(x: np.ndarray, dy: int, dx: int, padding: str = "circular") -> np.ndarray:
    """out[c, y, x] = in[c, y - dy, x - dx]: indices wrap ("circular") or read
    zero outside the field ("zero")."""
    if padding == "circular":
        return np.roll(x, (dy, dx), axis=(1, 2))
    out = np.zeros_like(x)
    H, W = x.shape[1:]
    ys, yd = (slice(0, H - dy), slice(dy, H)) if dy >= 0 else (slice(-dy, H), slice(0, H + dy))
    xs, xd = (slice(0, W - dx), slice(dx, W)) if dx >= 0 else (slice(-dx, W), slice(0, W + dx))
    out[:, yd, xd] = x[:, ys, xs]
    return out


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray, padding: str = "circular") -> np.ndarray:
    """out[o, y, x] = b[o] + sum_{c, ky, kx} w[o, c, ky, kx] in[c, y+ky-1, x+kx-1].

    Indices wrap (circular padding), or read zero outside the field (zero
    padding, for windows of a field).  Each of the nine taps is a shifted copy
    of the input contracted over channels.
    """
    cout = w.shape[0]
    out = np.broadcast_to(b[:, None, None], (cout,) + x.shape[1:]).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            shifted = shift2d(x, 1 - ky, 1 - kx, padding)
            out += np.einsum("oc,chw->ohw", w[:, :, ky, kx], shifted)
    return out


def prelu(x: np.ndarray, a: np.ndarray) -> np.ndarray:
    """y = x where x > 0, a_c x otherwise, one slope per channel."""
    return np.where(x > 0, x, a[:, None, None] * x)


def pixel_shuffle2(x: np.ndarray) -> np.ndarray:
    """(4C, H, W) -> (C, 2H, 2W): out[c, 2y+dy, 2x+dx] = in[4c + 2dy + dx, y, x]."""
    c4, H, W = x.shape
    c = c4 // 4
    out = np.empty((c, 2 * H, 2 * W))
    for dy in range(2):
        for dx in range(2):
            out[:, dy::2, dx::2] = x[np.arange(c) * 4 + 2 * dy + dx]
    return out


def generator_forward(q: np.ndarray, weights: dict, n_blocks: int = N_BLOCKS,
                      emulate_bf16: bool = False, padding: str = "circular") -> np.ndarray:
    """G(q) for a normalised coarse field q (H, W) -> fine field (2H, 2W);
    padding "zero" treats q as a window cut out of a larger field."""
    rnd = bf16_round if emulate_bf16 else (lambda a: a)
    W = {k: (rnd(v) if (emulate_bf16 and k.endswith(("w", "w1", "w2"))) else v)
         for k, v in weights.items()}
    x = q[None, :, :].astype(np.float64)
    x = rnd(prelu(conv3x3(x, W["in.w"], W["in.b"], padding), W["in.a"]))
    for k in range(n_blocks):
        t = rnd(prelu(conv3x3(x, W[f"b{k}.w1"], W[f"b{k}.b1"], padding), W[f"b{k}.a"]))
        x = rnd(x + conv3x3(t, W[f"b{k}.w2"], W[f"b{k}.b2"], padding))
    u = conv3x3(x, W["up.w"], W["up.b"], padding)
    u = rnd(prelu(pixel_shuffle2(u), W["up.a"]))
    return conv3x3(u, W["out.w"], W["out.b"], padding)[0]


def generator_stages(q: np.ndarray, weights: dict, n_blocks: int = N_BLOCKS,
                     emulate_bf16: bool = False, padding: str = "circular") -> list:
    """The layers of generator_forward one by one: a list of (v, a) per stage,
    v the stage's value before its output is stored and a the stored value
    (v rounded to bf16 with emulate_bf16, else v).  Stages: the 1 -> 64 layer
    with PReLU; for each residual block its first convolution with PReLU and
    its second convolution plus the skip; the 64 -> 256 layer with the pixel
    shuffle and PReLU; the 64 -> 1 layer (its a is v: the output is not
    stored as bf16).  Each stage reads the previous stage's a."""
    rnd = bf16_round if emulate_bf16 else (lambda a: a)
    W = {k: (rnd(v) if (emulate_bf16 and k.endswith(("w", "w1", "w2"))) else v)
         for k, v in weights.items()}
    out = []
    v = prelu(conv3x3(q[None, :, :].astype(np.float64), W["in.w"], W["in.b"], padding), W["in.a"])
    out.append((v, rnd(v)))
    for k in range(n_blocks):
        x = out[-1][1]
        v = prelu(conv3x3(x, W[f"b{k}.w1"], W[f"b{k}.b1"], padding), W[f"b{k}.a"])
        out.append((v, rnd(v)))
        v = x + conv3x3(out[-1][1], W[f"b{k}.w2"], W[f"b{k}.b2"], padding)
        out.append((v, rnd(v)))
    v = prelu(pixel_shuffle2(conv3x3(out[-1][1], W["up.w"], W["up.b"], padding)), W["up.a"])
    out.append((v, rnd(v)))
    v = conv3x3(out[-1][1], W["out.w"], W["out.b"], padding)[0]
    out.append((v, v))
    return out


def _conv3x3_valid(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """conv3x3 without padding: the output is 2 smaller in each direction and
    every value is the full 3x3 sum (no wrap, no zeros)."""
    cout = w.shape[0]
    H, W = x.shape[1] - 2, x.shape[2] - 2
    out = np.broadcast_to(b[:, None, None], (cout, H, W)).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,chw->ohw", w[:, :, ky, kx], x[:, ky:ky + H, kx:kx + W])
    return out


def generator_reach(n_blocks: int = N_BLOCKS) -> int:
    """Coarse cells around a fine point's coarse cell that its G value depends
    on: the first conv, two per residual block and the up conv at coarse
    resolution, plus one coarse cell for the last (fine) conv."""
    return 2 * n_blocks + 3


def generator_at(q: np.ndarray, weights: dict, points, n_blocks: int = N_BLOCKS,
                 emulate_bf16: bool = False) -> np.ndarray:
    """G(q) of a periodic coarse field q at the fine points [(Y, X), ...], each
    computed from its own neighbourhood of coarse cells (generator_reach
    around (Y // 2, X // 2), indices wrapped) with unpadded convolutions, so the
    cost per point does not depend on the grid size.  Same layers, order and
    bf16 rounding points as generator_forward."""
    rnd = bf16_round if emulate_bf16 else (lambda a: a)
    W = {k: (rnd(v) if (emulate_bf16 and k.endswith(("w", "w1", "w2"))) else v)
         for k, v in weights.items()}
    n = q.shape[0]
    R = generator_reach(n_blocks)
    if 2 * R + 1 > n:
        raise ValueError(f"grid {n} smaller than the generator's reach {2 * R + 1}")
    out = []
    for Y, X in points:
        cy, cx = Y // 2, X // 2
        rows = (cy - R + np.arange(2 * R + 1)) % n
        cols = (cx - R + np.arange(2 * R + 1)) % n
        x = q[np.ix_(rows, cols)][None, :, :].astype(np.float64)
        x = rnd(prelu(_conv3x3_valid(x, W["in.w"], W["in.b"]), W["in.a"]))
        for k in range(n_blocks):
            t = rnd(prelu(_conv3x3_valid(x, W[f"b{k}.w1"], W[f"b{k}.b1"]), W[f"b{k}.a"]))
            x = rnd(x[:, 2:-2, 2:-2] + _conv3x3_valid(t, W[f"b{k}.w2"], W[f"b{k}.b2"]))
        u = _conv3x3_valid(x, W["up.w"], W["up.b"])  # 3 x 3 coarse cells: cy - 1 .. cy + 1
        u = rnd(prelu(pixel_shuffle2(u), W["up.a"]))  # fine rows 2 cy - 2 .. 2 cy + 3
        g = _conv3x3_valid(u, W["out.w"], W["out.b"])[0]  # fine rows 2 cy - 1 .. 2 cy + 2
        out.append(g[Y - (2 * cy - 1), X - (2 * cx - 1)])
    return np.array(out)


def generator_block(q: np.ndarray, weights: dict, y0: int, x0: int, rows: int, cols: int,
                    n_blocks: int = N_BLOCKS, emulate_bf16: bool = False) -> np.ndarray:
    """G(q) of a periodic coarse field q on the block of fine points
    [y0, y0 + rows) x [x0, x0 + cols) (all even; the block may wrap around the
    grid), from the block's own neighbourhood of coarse cells (generator_reach
    beyond the block's coarse cells, indices wrapped) with unpadded
    convolutions.  The same computation as generator_at for every point of
    the block, sharing the layers' work between neighbouring points."""
    if y0 % 2 or x0 % 2 or rows % 2 or cols % 2 or rows <= 0 or cols <= 0:
        raise ValueError("block origin and size must be even and positive")
    rnd = bf16_round if emulate_bf16 else (lambda a: a)
    W = {k: (rnd(v) if (emulate_bf16 and k.endswith(("w", "w1", "w2"))) else v)
         for k, v in weights.items()}
    n = q.shape[0]
    R = generator_reach(n_blocks)
    if rows // 2 + 2 * R > n or cols // 2 + 2 * R > n:
        raise ValueError("block and the generator's reach exceed the grid")
    ridx = (y0 // 2 - R + np.arange(rows // 2 + 2 * R)) % n
    cidx = (x0 // 2 - R + np.arange(cols // 2 + 2 * R)) % n
    x = q[np.ix_(ridx, cidx)][None, :, :].astype(np.float64)
    x = rnd(prelu(_conv3x3_valid(x, W["in.w"], W["in.b"]), W["in.a"]))
    for k in range(n_blocks):
        t = rnd(prelu(_conv3x3_valid(x, W[f"b{k}.w1"], W[f"b{k}.b1"]), W[f"b{k}.a"]))
        x = rnd(x[:, 2:-2, 2:-2] + _conv3x3_valid(t, W[f"b{k}.w2"], W[f"b{k}.b2"]))
    u = _conv3x3_valid(x, W["up.w"], W["up.b"])  # coarse cells y0/2 - 1 .. (y0 + rows)/2
    u = rnd(prelu(pixel_shuffle2(u), W["up.a"]))  # fine rows y0 - 2 .. y0 + rows + 1
    g = _conv3x3_valid(u, W["out.w"], W["out.b"])[0]  # fine rows y0 - 1 .. y0 + rows
    return g[1:rows + 1, 1:cols + 1]


def sr_scale(ec: np.ndarray) -> float:
    """Input scale s = max |e_c|, or 1 for a zero field."""
    s = float(np.max(np.abs(ec)))
    return s if s > 0.0 else 1.0


def sr_prolong(ec: np.ndarray, weights: dict, n_blocks: int = N_BLOCKS,
               emulate_bf16: bool = False) -> np.ndarray:
    """SR prolongation e_f = P_cubic e_c + s G(e_c / s)."""
    s = sr_scale(ec)
    q = ec / s
    if emulate_bf16:
        q = np.asarray(q, dtype=np.float32).astype(np.float64)
    return prolong_cubic(ec) + s * generator_forward(q, weights, n_blocks, emulate_bf16)
