"""Parity of the windowed SR prolongation (Sec. 3.1, Fig. 2; Appendix A,
Algorithms 1-5) on the GPU against the oracle's windowed_sr_prolong (GPU).

The GPU lays the 6 x 6 windows out as a mosaic for its tensor-core
convolutions and runs the generator's layers with bf16 activations and FP32
accumulation; the oracle super-resolves every window on its own with zero
padding (oracle generator_forward with bf16 emulation) and stitches the kept
central blocks.  The comparison is made in the normalised domain: the
generator value g behind each fine output p = sgn(g) 10^(log10 p_min +
|g| (log10 p_max - log10 p_min)) is recovered exactly from the GPU's output.

Bound, element by element: the first-order propagation of the per-layer
error bounds through each window's network (as in test_gpu_sr_fullsize:
2^-8 |v| + max(1, |a|) K 2^-23 S at every stored value, times the absolute
derivative of the kept output with respect to it, by torch's CPU autograd in
FP64), plus the FP32 symmetric logarithm of the inputs (log10f, within 4e-7
of the normalised value) through the first layer.  With one residual block
the bound is tight; with the eight blocks of the trained generator it is
loose, and the outputs are also held to 0.1 max|g|.
"""
import numpy as np
import pytest

from oracle import generator as og
from oracle import windowed as ow
from synthetic.sources import turbulent_source
from synthetic.weights import random_weights

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U23 = 2.0 ** -23
P_MIN, P_MAX = 1e-10, 1e-3


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _windows(q, n_s=6, core=2):
    """Every window of the oracle's layout, (n/2)^2 x 6 x 6, in (a, b) order."""
    n = q.shape[0]
    m = (n_s - core) // 2
    idx = np.arange(n_s)
    out = []
    for a in range(n // core):
        rows = (core * a - m + idx) % n
        for b in range(n // core):
            out.append(q[np.ix_(rows, (core * b - m + idx) % n)])
    return np.array(out)


def _window_bound(wins, w, n_blocks):
    """First-order bound on |g_gpu - g| at the kept 4 x 4 points of every
    window (windows, 4, 4), by torch autograd over the batch of windows."""
    F = torch.nn.functional
    d = {k: torch.from_numpy(np.asarray(og.bf16_round(v) if k.endswith(("w", "w1", "w2")) else v, dtype=np.float64))
         for k, v in w.items()}
    one = torch.ones(1, dtype=torch.float64)

    def conv(x, wk, bk):
        return F.conv2d(x, d[wk], d[bk], padding=1)

    def S(x, wk, bk):
        return F.conv2d(x.detach().abs(), d[wk].abs(), d[bk].abs(), padding=1)

    def slope(a):
        return torch.maximum(a.abs(), one)[None, :, None, None]

    out = np.zeros((len(wins), 4, 4))
    for o in range(16):
        oy, ox = o // 4, o % 4
        x0 = torch.from_numpy(wins)[:, None].clone().requires_grad_(True)
        vs, eps = [], []
        v = F.prelu(conv(x0, "in.w", "in.b"), d["in.a"])
        eq = 4e-7 * F.conv2d(torch.ones_like(x0.detach()), d["in.w"].abs(), padding=1)  # FP32 symlog of the inputs
        eps.append(2.0 ** -8 * v.detach().abs() + (11 * U23 * S(x0, "in.w", "in.b") + eq) * slope(d["in.a"]))
        vs.append(v)
        x = v
        for k in range(n_blocks):
            t = F.prelu(conv(x, f"b{k}.w1", f"b{k}.b1"), d[f"b{k}.a"])
            eps.append(2.0 ** -8 * t.detach().abs() + 577 * U23 * S(x, f"b{k}.w1", f"b{k}.b1") * slope(d[f"b{k}.a"]))
            vs.append(t)
            y = x + conv(t, f"b{k}.w2", f"b{k}.b2")
            eps.append(2.0 ** -8 * y.detach().abs()
                       + 578 * U23 * (S(t, f"b{k}.w2", f"b{k}.b2") + x.detach().abs()))
            vs.append(y)
            x = y
        u = F.prelu(F.pixel_shuffle(conv(x, "up.w", "up.b"), 2), d["up.a"])
        eps.append(2.0 ** -8 * u.detach().abs()
                   + 577 * U23 * F.pixel_shuffle(S(x, "up.w", "up.b"), 2) * slope(d["up.a"]))
        vs.append(u)
        for v in vs:
            v.retain_grad()
        g = F.conv2d(u, d["out.w"], d["out.b"], padding=1)[:, 0, 4 + oy, 4 + ox]
        last = 578 * U23 * S(u, "out.w", "out.b")[:, 0, 4 + oy, 4 + ox].numpy()
        g.sum().backward()
        b = sum((v.grad.abs() * e).sum(dim=(1, 2, 3)).numpy() for v, e in zip(vs, eps))
        out[:, oy, ox] = b + last + 1e-7
    return out


def _stitch(per_window, n):
    """(n/2)^2 x 4 x 4 kept blocks -> 2n x 2n field, window (a, b) at rows 4a.., cols 4b.."""
    h = n // 2
    return per_window.reshape(h, h, 4, 4).transpose(0, 2, 1, 3).reshape(2 * n, 2 * n)


CASES = [(32, 1, "random"), (64, 1, "random"), (32, 8, "trained")]


@pytest.mark.parametrize("nc,n_blocks,kind", CASES, ids=[f"{c[0]}-{c[1]}blk-{c[2]}" for c in CASES])
def test_windowed_sr_matches_oracle(mg, nc, n_blocks, kind):
    from paper_2403_07936_gb300 import sr
    if kind == "trained":
        import os
        blob = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                 "paper_2403_07936_gb300", "weights", "sr_generator.mgsrw"), "rb").read()
        w = sr.unpack_weights(blob)
    else:
        w = random_weights(40 + nc, n_blocks=n_blocks, gain=0.5)
        blob = sr.pack_weights(w)
    ctx = mg.Context(int(np.log2(2 * nc // 8)) + 1, 2 * nc)
    ctx.load_weights(blob)
    # an error field spanning the normalisation interval: magnitudes 1e-9 .. 1e-4, both signs
    base = turbulent_source(nc, nc // 4, 71 + nc)
    ec = (np.sign(base) * np.power(10.0, -9 + 5 * np.abs(base) / np.abs(base).max())).astype(np.float32)
    ec[3, 5] = 0.0
    ect = torch.tensor(ec, device=DEV)
    out = torch.full((2 * nc, 2 * nc), float("nan"), dtype=torch.float32, device=DEV)
    mg.op_sr_windowed(ctx, ect, out, P_MIN, P_MAX)
    torch.cuda.synchronize()
    p = out.double().cpu().numpy()
    assert np.all(np.isfinite(p))
    lmin, span = np.log10(P_MIN), np.log10(P_MAX) - np.log10(P_MIN)
    g_gpu = np.where(p == 0, 0.0, np.sign(p) * (np.log10(np.abs(np.where(p == 0, 1.0, p))) - lmin) / span)
    q = ow.symlog_normalize(ec.astype(np.float64), P_MIN, P_MAX)
    gen = lambda win: og.generator_forward(win, w, n_blocks, emulate_bf16=True, padding="zero")  # noqa: E731
    g_ref = ow.windowed_upsample(q, gen, 2)
    # the oracle's full pipeline (normalise, windows, stitch, map back) is the same field
    np.testing.assert_allclose(ow.windowed_sr_prolong(ec.astype(np.float64), gen, 2, P_MIN, P_MAX),
                               ow.symlog_denormalize(g_ref, P_MIN, P_MAX), rtol=1e-12)
    bound = _stitch(_window_bound(_windows(q), w, n_blocks), nc)
    d = np.abs(g_gpu - g_ref)
    assert (d <= bound).all(), (float((d / bound).max()), float(d.max()))
    if n_blocks == 1:
        assert d.max() <= 2e-2 * np.abs(g_ref).max()
    else:
        assert d.max() <= 0.1 * np.abs(g_ref).max()


def test_windowed_sr_rejects_bad_arguments(mg):
    from paper_2403_07936_gb300 import sr
    ctx = mg.Context(6, 256)
    ec = torch.zeros((64, 64), dtype=torch.float32, device=DEV)
    out = torch.zeros((128, 128), dtype=torch.float32, device=DEV)
    with pytest.raises(mg.MGError) as e:
        mg.op_sr_windowed(ctx, ec, out)
    assert e.value.status == 6  # no weights
    ctx.load_weights(sr.pack_weights(random_weights(3, n_blocks=1)))
    with pytest.raises(mg.MGError) as e:
        mg.op_sr_windowed(ctx, ec, out, 1e-3, 1e-10)
    assert e.value.status == 1
    small = torch.zeros((16, 16), dtype=torch.float32, device=DEV)
    with pytest.raises(mg.MGError) as e:
        mg.op_sr_windowed(ctx, small, out)
    assert e.value.status == 1
