"""Seeded random generator weights (inputs for parity tests, not a trained model).

Parameter names and shapes follow the one-channel SR generator: conv3x3 1->64
with PReLU, residual blocks of two 64->64 conv3x3 with a PReLU between them,
conv3x3 64->256 followed by pixel-shuffle x2 and PReLU, and conv3x3 64->1.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 64
N_BLOCKS = 8


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


def random_weights(seed: int, n_feat: int = N_FEAT, n_blocks: int = N_BLOCKS,
                   gain: float = 1.0) -> dict:
    """He-style random weights drawn from numpy's PCG64 with the given seed."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, shape in weight_shapes(n_feat, n_blocks):
        if name.endswith((".w", ".w1", ".w2")):
            fan_in = shape[1] * 9
            out[name] = rng.standard_normal(shape) * gain * np.sqrt(2.0 / fan_in)
        elif name.endswith(".a"):
            out[name] = rng.uniform(0.05, 0.3, size=shape)
        else:
            out[name] = rng.standard_normal(shape) * 0.05
    return out
