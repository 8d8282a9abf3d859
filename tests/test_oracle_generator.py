"""Pins of the SR-generator oracle against PyTorch's CPU library routines
(conv2d with circular padding, pixel_shuffle, prelu, bfloat16 casts) in FP64,
and against closed-form special cases (no GPU)."""
import numpy as np
import pytest

from oracle import generator as g
from oracle import multigrid as mg
from synthetic.weights import random_weights

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _tconv(x, w, b):
    return F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), torch.tensor(w), torch.tensor(b))


def test_conv3x3_matches_torch_circular():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 7, 9))
    w = rng.standard_normal((6, 5, 3, 3))
    b = rng.standard_normal(6)
    ref = _tconv(torch.tensor(x)[None], w, b)[0].numpy()
    np.testing.assert_allclose(g.conv3x3(x, w, b), ref, atol=1e-12)


def test_conv3x3_delta_kernel_is_shift():
    """A single unit tap at (ky, kx) reads in[y + ky - 1, x + kx - 1] (wrapped)."""
    x = np.random.default_rng(1).standard_normal((1, 6, 8))
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 2, 0] = 1.0  # ky=2 -> y+1, kx=0 -> x-1
    out = g.conv3x3(x, w, np.zeros(1))
    np.testing.assert_array_equal(out[0], np.roll(x[0], (-1, 1), axis=(0, 1)))


def test_pixel_shuffle_matches_torch():
    x = np.random.default_rng(2).standard_normal((12, 4, 5))
    ref = F.pixel_shuffle(torch.tensor(x)[None], 2)[0].numpy()
    np.testing.assert_array_equal(g.pixel_shuffle2(x), ref)


def test_generator_matches_torch_composition():
    w = random_weights(3, n_feat=8, n_blocks=2)
    q = np.random.default_rng(4).standard_normal((6, 10))
    T = torch.tensor
    x = T(q)[None, None]
    x = F.prelu(_tconv(x, w["in.w"], w["in.b"]), T(w["in.a"]))
    for k in range(2):
        t = F.prelu(_tconv(x, w[f"b{k}.w1"], w[f"b{k}.b1"]), T(w[f"b{k}.a"]))
        x = x + _tconv(t, w[f"b{k}.w2"], w[f"b{k}.b2"])
    u = F.prelu(F.pixel_shuffle(_tconv(x, w["up.w"], w["up.b"]), 2), T(w["up.a"]))
    ref = _tconv(u, w["out.w"], w["out.b"])[0, 0].numpy()
    np.testing.assert_allclose(g.generator_forward(q, w, n_blocks=2), ref, atol=1e-12)


def test_bf16_round_matches_torch_cast():
    a = np.random.default_rng(5).standard_normal(10000) * 10.0 ** np.random.default_rng(6).integers(-8, 8, 10000)
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(g.bf16_round(a), ref)


def test_sr_prolong_with_zero_generator_is_cubic():
    w = {k: np.zeros_like(v) for k, v in random_weights(7, n_feat=8, n_blocks=1).items()}
    ec = np.random.default_rng(8).standard_normal((8, 8))
    np.testing.assert_allclose(g.sr_prolong(ec, w, n_blocks=1), mg.prolong_cubic(ec), atol=0)


def test_sr_prolong_scale_equivariance():
    """s = max|e_c| makes the SR prolongation positively homogeneous."""
    w = random_weights(9, n_feat=8, n_blocks=1)
    ec = np.random.default_rng(10).standard_normal((8, 8))
    a = g.sr_prolong(ec, w, n_blocks=1)
    b = g.sr_prolong(1e-6 * ec, w, n_blocks=1)
    np.testing.assert_allclose(b, 1e-6 * a, rtol=1e-10, atol=1e-20)
    assert g.sr_scale(np.zeros((4, 4))) == 1.0


def test_sampled_generator_equals_the_whole_grid_forward_pass():
    """generator_at (unpadded convolutions on each point's neighbourhood) gives
    the whole-grid circular forward pass's values at those points, plain and
    with bf16 emulation, including points whose neighbourhood wraps."""
    from oracle import generator as og
    from synthetic.weights import random_weights
    w = random_weights(3)
    q = np.random.default_rng(0).standard_normal((48, 48))
    pts = [(0, 0), (95, 95), (1, 94), (47, 50), (10, 3), (60, 91), (33, 0)]
    for bf16 in (False, True):
        full = og.generator_forward(q, w, emulate_bf16=bf16)
        got = og.generator_at(q, w, pts, emulate_bf16=bf16)
        np.testing.assert_array_equal(got, np.array([full[y, x] for y, x in pts]))


def test_generator_reach_is_tight():
    """A fine point's value depends on coarse cells up to generator_reach away
    (on the side its fine-grid parity faces) and on none further."""
    from oracle import generator as og
    from synthetic.weights import random_weights
    nb, n = 2, 32
    w = random_weights(3, n_blocks=nb)
    q = np.random.default_rng(0).standard_normal((n, n))
    R = og.generator_reach(nb)
    for Y, side in ((20, -1), (21, +1)):  # even fine rows reach further up, odd ones further down
        cy, cx = Y // 2, 21 // 2
        base = og.generator_forward(q, w, n_blocks=nb)[Y, 21]

        def bumped(d):
            q2 = q.copy()
            q2[(cy + d) % n, cx] += 1.0
            return og.generator_forward(q2, w, n_blocks=nb)[Y, 21]

        assert bumped(side * R) != base
        assert bumped(side * (R + 1)) == base and bumped(-side * R) == base


def test_block_generator_equals_the_whole_grid_forward_pass():
    """generator_block (one unpadded neighbourhood for a block of fine points)
    gives the whole-grid circular forward pass's values on the block, plain and
    with bf16 emulation, for blocks inside the grid and blocks that wrap
    around its edges and corner."""
    from oracle import generator as og
    from synthetic.weights import random_weights
    w = random_weights(3)
    q = np.random.default_rng(0).standard_normal((48, 48))
    nf = 96
    for bf16 in (False, True):
        full = og.generator_forward(q, w, emulate_bf16=bf16)
        for y0, x0, rows, cols in ((0, 0, 8, 8), (40, 12, 6, 10), (92, 90, 8, 10), (94, 0, 4, 6)):
            got = og.generator_block(q, w, y0, x0, rows, cols, emulate_bf16=bf16)
            ref = full[np.ix_((y0 + np.arange(rows)) % nf, (x0 + np.arange(cols)) % nf)]
            np.testing.assert_array_equal(got, ref)
    with pytest.raises(ValueError):
        og.generator_block(q, w, 1, 0, 4, 4)


def test_generator_stages_compose_to_the_forward_pass():
    """generator_stages: each stage is the stated layer of the previous
    stage's stored output (checked against torch's conv2d, prelu and
    pixel_shuffle for the first and the shuffle stage), the stored values are
    the bf16 roundings, and the last stage is generator_forward bit for bit."""
    from oracle import generator as og
    w = random_weights(5)
    q = np.random.default_rng(1).standard_normal((16, 16))
    for bf16 in (False, True):
        st = og.generator_stages(q, w, emulate_bf16=bf16)
        assert len(st) == 2 * og.N_BLOCKS + 3
        np.testing.assert_array_equal(st[-1][0], og.generator_forward(q, w, emulate_bf16=bf16))
        for v, a in st[:-1]:
            np.testing.assert_array_equal(a, g.bf16_round(v) if bf16 else v)
    st = og.generator_stages(q, w)
    x = torch.from_numpy(np.pad(q, 1, mode="wrap"))[None, None]
    ref = F.prelu(F.conv2d(x, torch.from_numpy(w["in.w"]), torch.from_numpy(w["in.b"])),
                  torch.from_numpy(w["in.a"]))[0].numpy()
    np.testing.assert_allclose(st[0][0], ref, rtol=1e-12, atol=1e-12)
    a = torch.from_numpy(np.pad(st[-3][1], ((0, 0), (1, 1), (1, 1)), mode="wrap"))[None]
    u = F.conv2d(a, torch.from_numpy(w["up.w"]), torch.from_numpy(w["up.b"]))
    ref = F.prelu(F.pixel_shuffle(u, 2), torch.from_numpy(w["up.a"]))[0].numpy()
    np.testing.assert_allclose(st[-2][0], ref, rtol=1e-12, atol=1e-12)
