"""Element-wise parity of the SR generator, layer by layer, at the grid sizes
of the SR workloads (1024^2 and 2048^2 fine grids) with the trained weights,
and of the composed generator at sampled points (GPU).

Layers.  Each layer of the generator (Sec. 2.3, Fig. 1b; Appendix A,
Algorithm 5) runs through mg_op_sr_layer - the production kernel with the
context's packed trained weights - on an input the oracle computed: the
oracle's own stage chain (bf16-emulating) on a 128^2 coarse error, tiled
periodically to the full coarse grid (512^2 or 1024^2), which is again a
periodic field, so the exact layer output is the tiled oracle output at every
point of the full grid.  Every point of every layer is compared with the a
priori bound

    |gpu - ref| <= 2^-8 |ref| + (1 + 2^-7) max(1, |a|) K 2^-23 S

where 2^-8 |ref| is half a bf16 spacing (the output is rounded to bf16 once),
K 2^-23 S bounds an FP32 accumulation of K terms of absolute sum S (products
of bf16 values are exact in FP32; each addition, rounded or truncated, errs
by at most 2^-23 of the running sum), and a is the PReLU slope (a value whose
sign flips inside that error is scaled by a).  The CUDA-core layers (1 -> 64
on ec / s, 64 -> 1 times s) and s = max|ec| are checked the same way (s
exactly).  The chain of the GPU's layers is then shown to be the production
generator bit for bit.

Composition.  The generator with the trained weights on real 512^2 and
1024^2 coarse errors is compared element by element with the oracle's
bf16-emulating and FP64 forward passes (oracle generator_at at 64 sampled
fine points, generator_block on blocks of 2048 fine points, blocks and
points wrapping around the grid's corner).  The GPU and the oracle round
different values to bf16 wherever their sums differ near a rounding
boundary, and each layer's own error (within the bound above) travels
through the later layers.  The derived bound is that propagation to first
order: the layer bound eps of every stored value times the absolute
derivative of the output with respect to it (the output's Jacobian, taken by
torch's CPU autograd in FP64 on the point's neighbourhood), summed.  It
assumes every stored value errs the worst way at once and comes to 0.7 to 4
times max|G|; the measured differences are 2 to 4 % of max|G|, so the blocks
also hold a tighter check, 0.1 max|ref| element by element.
"""
import os

import numpy as np
import pytest

from oracle import generator as og
from oracle import multigrid as omg
from synthetic.sources import config_seed, turbulent_source

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U23 = 2.0 ** -23
M = 128  # coarse size of the oracle's stage chain (tiled to the full size)
NB = og.N_BLOCKS
TRAINED = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2403_07936_gb300",
                       "weights", "sr_generator.mgsrw")


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _trained():
    from paper_2403_07936_gb300 import sr
    blob = open(TRAINED, "rb").read()
    return blob, sr.unpack_weights(blob)


def _coarse_error(nf, seed):
    """A coarse-grid error of the kind the finest transition sees: the exact
    coarse solution of the fully weighted turbulent source (FP32)."""
    f = turbulent_source(nf, nf // 8, seed)
    rc = omg.restrict_fw(f - f.mean())
    return omg.exact_solve_fft(rc - rc.mean(), omg.grid_h(nf // 2)).astype(np.float32)


def _abs_conv(x, w, b):
    """S = |b| + sum |w| |x| over each output's 3 x 3 x C window (circular)."""
    return og.conv3x3(np.abs(x), np.abs(w), np.abs(b))


@pytest.fixture(scope="module")
def chain():
    """The oracle's stage chain on a 128^2 coarse error with the trained
    weights (bf16 emulation), with the absolute sums S of every stage."""
    _, w = _trained()
    W = {k: (og.bf16_round(v) if k.endswith(("w", "w1", "w2")) else v) for k, v in w.items()}
    ec = _coarse_error(2 * M, config_seed(2, 0)).astype(np.float64)
    s = og.sr_scale(ec)
    q = ec / s
    st = og.generator_stages(q, w, emulate_bf16=True)
    S = [_abs_conv(q[None], W["in.w"], W["in.b"])]
    for k in range(NB):
        S.append(_abs_conv(st[2 * k][1], W[f"b{k}.w1"], W[f"b{k}.b1"]))
        S.append(_abs_conv(st[2 * k + 1][1], W[f"b{k}.w2"], W[f"b{k}.b2"]) + np.abs(st[2 * k][1]))
    S.append(og.pixel_shuffle2(_abs_conv(st[2 * NB][1], W["up.w"], W["up.b"])))
    S.append(s * _abs_conv(st[2 * NB + 1][1], W["out.w"], W["out.b"])[0])
    slopes = [W["in.a"]] + sum(([W[f"b{k}.a"], np.ones(64)] for k in range(NB)), []) + [W["up.a"], np.ones(1)]
    return {"ec": ec, "s": s, "stages": st, "S": S, "slopes": slopes}


def _to_dev(a_chw, reps):
    """(C, m, m) oracle activation -> padded, tiled (reps m + 2)^2 x C bf16 on the device."""
    t = np.tile(a_chw.transpose(1, 2, 0), (reps, reps, 1))
    t = np.pad(t, ((1, 1), (1, 1), (0, 0)), mode="wrap")
    return torch.tensor(t, dtype=torch.float32, device=DEV).to(torch.bfloat16)


def _compare_tiled(got, ref, S, K, slope, m):
    """got: (n, n[, C]) float64 host array, n a multiple of m; ref and S the
    oracle's (C, m, m) or (m, m) arrays; every point of every tile."""
    if ref.ndim == 3:
        ref, S = ref.transpose(1, 2, 0), S.transpose(1, 2, 0)
    n = got.shape[0]
    tol = 2.0 ** -8 * np.abs(ref) + (1 + 2.0 ** -7) * np.maximum(1.0, np.abs(slope)) * K * U23 * S
    for ty in range(n // m):
        band = got[ty * m:(ty + 1) * m].reshape((m, n // m, m) + got.shape[2:]).swapaxes(0, 1)
        d = np.abs(band - ref[None])
        bad = d > tol[None]
        assert not bad.any(), (ty, int(bad.sum()), float(d.max()))


def _halo_ok(a, n):
    a16 = a.view(torch.int16)
    inner = a16[1:n + 1, 1:n + 1]
    assert torch.equal(a16[0, 1:n + 1], inner[n - 1]) and torch.equal(a16[n + 1, 1:n + 1], inner[0])
    assert torch.equal(a16[:, 0], a16[:, n]) and torch.equal(a16[:, n + 1], a16[:, 1])


@pytest.mark.parametrize("nc", [128, 512, 1024])
def test_generator_layers_elementwise(mg, chain, nc):
    blob, _ = _trained()
    nf = 2 * nc
    reps = nc // M
    ctx = mg.Context(int(np.log2(nf // 8)) + 1, nf)
    ctx.load_weights(blob)
    st, S, slopes = chain["stages"], chain["S"], chain["slopes"]

    # layer 0: s = max|ec| and PReLU(conv 1 -> 64 of ec / s)
    ect = torch.tensor(np.tile(chain["ec"], (reps, reps)), dtype=torch.float32, device=DEV)
    s_dev = torch.zeros(1, dtype=torch.float32, device=DEV)
    out = torch.full((nc + 2, nc + 2, 64), float("nan"), dtype=torch.bfloat16, device=DEV)
    mg.op_sr_layer(ctx, 0, nc, ect, out, s_dev)
    torch.cuda.synchronize()
    assert s_dev.item() == chain["s"]
    _compare_tiled(out[1:-1, 1:-1].double().cpu().numpy(), st[0][0], S[0], 11, slopes[0], M)
    _halo_ok(out, nc)

    # block layers and the pixel-shuffle layer, each on the oracle's previous stage
    for layer in range(1, 2 * NB + 2):
        inp = _to_dev(st[layer - 1][1], reps)
        skip = _to_dev(st[layer - 2][1], reps) if (layer <= 2 * NB and layer % 2 == 0) else None
        n_out = nf if layer == 2 * NB + 1 else nc
        out = torch.full((n_out + 2, n_out + 2, 64), float("nan"), dtype=torch.bfloat16, device=DEV)
        mg.op_sr_layer(ctx, layer, nc, inp, out, s_dev, skip=skip)
        torch.cuda.synchronize()
        K = 578 if skip is not None else 577
        m = 2 * M if layer == 2 * NB + 1 else M
        _compare_tiled(out[1:-1, 1:-1].double().cpu().numpy(), st[layer][0], S[layer], K, slopes[layer], m)
        _halo_ok(out, n_out)

    # layer 2 NB + 2: s * conv 64 -> 1 (FP32 output, s = the oracle's scale)
    inp = _to_dev(st[2 * NB + 1][1], reps)
    s_in = torch.tensor([chain["s"]], dtype=torch.float32, device=DEV)
    out = torch.full((nf, nf), float("nan"), dtype=torch.float32, device=DEV)
    mg.op_sr_layer(ctx, 2 * NB + 2, nc, inp, out, s_in)
    torch.cuda.synchronize()
    ref = chain["s"] * st[-1][0]
    got = out.double().cpu().numpy()
    tol = 2 * 2.0 ** -24 * np.abs(ref) + 578 * U23 * S[-1]
    for ty in range(nf // (2 * M)):
        band = got[ty * 2 * M:(ty + 1) * 2 * M].reshape(2 * M, nf // (2 * M), 2 * M).swapaxes(0, 1)
        assert not (np.abs(band - ref[None]) > tol[None]).any(), ty


@pytest.mark.parametrize("nc", [512, 1024])
def test_generator_is_the_chain_of_its_layers(mg, nc):
    """mg_op_sr_generator equals the chain of mg_op_sr_layer calls bit for bit
    on a real coarse error of the full size, and s = max|ec| exactly."""
    blob, _ = _trained()
    nf = 2 * nc
    ctx = mg.Context(int(np.log2(nf // 8)) + 1, nf)
    ctx.load_weights(blob)
    ec = _coarse_error(nf, config_seed(2, nc))
    ect = torch.tensor(ec, device=DEV)
    s = torch.zeros(1, dtype=torch.float32, device=DEV)
    acts = [torch.empty((nc + 2, nc + 2, 64), dtype=torch.bfloat16, device=DEV) for _ in range(3)]
    mg.op_sr_layer(ctx, 0, nc, ect, acts[0], s)
    assert s.item() == float(np.abs(ec).max())
    cur = 0
    for k in range(NB):
        t, nxt = (cur + 1) % 3, (cur + 2) % 3
        mg.op_sr_layer(ctx, 2 * k + 1, nc, acts[cur], acts[t], s)
        mg.op_sr_layer(ctx, 2 * k + 2, nc, acts[t], acts[nxt], s, skip=acts[cur])
        cur = nxt
    fine = torch.empty((nf + 2, nf + 2, 64), dtype=torch.bfloat16, device=DEV)
    mg.op_sr_layer(ctx, 2 * NB + 1, nc, acts[cur], fine, s)
    chained = torch.empty((nf, nf), dtype=torch.float32, device=DEV)
    mg.op_sr_layer(ctx, 2 * NB + 2, nc, fine, chained, s)
    full = torch.empty((nf, nf), dtype=torch.float32, device=DEV)
    mg.op_sr_generator(ctx, ect, full)
    torch.cuda.synchronize()
    assert torch.equal(full, chained)


def _propagated_bound(q, w, points):
    """First-order element-wise error bound of the generator at fine points
    [(Y, X), ...]: each stage's stored output may differ from its exact value
    by eps = 2^-8 |v| + max(1, |a|) K 2^-23 S (the layer bound above), and
    the output's sensitivity to every stored value is the absolute Jacobian,
    so |G_gpu - G| <= sum over stages and values of |dG/dv| eps (plus the
    last layer's own accumulation error).  The Jacobian is taken by torch's
    CPU autograd (FP64) on each point's neighbourhood (generator_reach)."""
    F = torch.nn.functional
    d = {k: torch.from_numpy(np.asarray(og.bf16_round(v) if k.endswith(("w", "w1", "w2")) else v, dtype=np.float64))
         for k, v in w.items()}
    one = torch.ones(1, dtype=torch.float64)
    n = q.shape[0]
    R = og.generator_reach()

    def S(x, wk, bk):
        return F.conv2d(x.detach().abs(), d[wk].abs(), d[bk].abs())

    def slope(a):
        return torch.maximum(a.abs(), one)[None, :, None, None]

    out = []
    for Y, X in points:
        cy, cx = Y // 2, X // 2
        rows, cols = (cy - R + np.arange(2 * R + 1)) % n, (cx - R + np.arange(2 * R + 1)) % n
        x0 = torch.from_numpy(q[np.ix_(rows, cols)])[None, None].clone().requires_grad_(True)
        vs, eps = [], []
        v = F.prelu(F.conv2d(x0, d["in.w"], d["in.b"]), d["in.a"])
        eps.append(2.0 ** -8 * v.detach().abs() + 11 * U23 * S(x0, "in.w", "in.b") * slope(d["in.a"]))
        vs.append(v)
        x = v
        for k in range(NB):
            t = F.prelu(F.conv2d(x, d[f"b{k}.w1"], d[f"b{k}.b1"]), d[f"b{k}.a"])
            eps.append(2.0 ** -8 * t.detach().abs() + 577 * U23 * S(x, f"b{k}.w1", f"b{k}.b1") * slope(d[f"b{k}.a"]))
            vs.append(t)
            y = x[:, :, 2:-2, 2:-2] + F.conv2d(t, d[f"b{k}.w2"], d[f"b{k}.b2"])
            eps.append(2.0 ** -8 * y.detach().abs()
                       + 578 * U23 * (S(t, f"b{k}.w2", f"b{k}.b2") + x.detach()[:, :, 2:-2, 2:-2].abs()))
            vs.append(y)
            x = y
        u = F.prelu(F.pixel_shuffle(F.conv2d(x, d["up.w"], d["up.b"]), 2), d["up.a"])
        eps.append(2.0 ** -8 * u.detach().abs()
                   + 577 * U23 * F.pixel_shuffle(S(x, "up.w", "up.b"), 2) * slope(d["up.a"]))
        vs.append(u)
        for v in vs:
            v.retain_grad()
        iy, ix = Y - (2 * cy - 1), X - (2 * cx - 1)
        g = F.conv2d(u, d["out.w"], d["out.b"])[0, 0, iy, ix]
        last = 578 * U23 * float(S(u, "out.w", "out.b")[0, 0, iy, ix])
        g.backward()
        out.append(sum(float((v.grad.abs() * e).sum()) for v, e in zip(vs, eps)) + last)
    return np.array(out)


@pytest.mark.parametrize("nc", [512, 1024])
def test_generator_end_to_end_elementwise(mg, nc):
    """The composed generator with the trained weights against the oracle's
    bf16-emulating and FP64 forward passes, element by element: at 64 sampled
    fine points (corners included) within the first-order propagated bound of
    the layer errors, and on blocks of 2048 fine points within 0.1 max|ref|
    (measured: 0.039 at 512^2 coarse, 0.020 at 1024^2; the propagated bound
    is 0.7 to 4 max|G|, loose because it lets every stored value err the same
    way)."""
    blob, w = _trained()
    nf = 2 * nc
    ctx = mg.Context(int(np.log2(nf // 8)) + 1, nf)
    ctx.load_weights(blob)
    ec = _coarse_error(nf, config_seed(2, nc + 1))
    ect = torch.tensor(ec, device=DEV)
    out = torch.empty((nf, nf), dtype=torch.float32, device=DEV)
    mg.op_sr_generator(ctx, ect, out)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    s = og.sr_scale(ec.astype(np.float64))
    q = ec.astype(np.float64) / s
    rng = np.random.default_rng(nc)
    pts = [(0, 0), (nf - 1, nf - 1), (0, nf - 1), (nf - 1, 0)] + [tuple(int(v) for v in p)
                                                                  for p in rng.integers(0, nf, (60, 2))]
    ref = s * og.generator_at(q, w, pts, emulate_bf16=True)
    ref64 = s * og.generator_at(q, w, pts)
    bound = s * _propagated_bound(q, w, pts)
    g = np.array([got[y, x] for y, x in pts])
    assert (np.abs(g - ref) <= bound).all(), np.max(np.abs(g - ref) / bound)
    assert (np.abs(g - ref64) <= 2 * bound).all(), np.max(np.abs(g - ref64) / bound)
    blocks = [(nf - 16, nf - 8), (0, nf // 2), (nf // 2 + 2, 6), (nf // 4, 3 * nf // 4)]
    for y0, x0 in blocks:
        ref = s * og.generator_block(q, w, y0, x0, 32, 16, emulate_bf16=True)
        gb = got[np.ix_((y0 + np.arange(32)) % nf, (x0 + np.arange(16)) % nf)]
        scale = np.abs(ref).max()
        assert np.abs(gb - ref).max() <= 0.1 * scale, np.abs(gb - ref).max() / scale
