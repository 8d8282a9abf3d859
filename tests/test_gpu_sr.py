"""Parity of the super-resolution prolongation against the FP64 generator
oracle (GPU).

Each tensor-core convolution layer is compared with the FP64 convolution of
the same bf16 inputs and weights: the kernel accumulates in FP32 and rounds
its output to bf16 once, so the bound is half a bf16 spacing (2^-8 relative)
plus FP32 accumulation error (1e-5 of the layer's largest output).  The full
generator is compared with the oracle's bf16-emulating forward pass in
relative L2 norm (a bf16 rounding that lands on the other side of a tie
propagates, so element-wise equality is not expected).
"""
import numpy as np
import pytest

from oracle import generator as og
from oracle import multigrid as omg
from synthetic.sources import turbulent_source
from synthetic.weights import random_weights

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _pad(a):
    """(H, W, C) -> (H+2, W+2, C) with periodic halo."""
    return np.pad(a, ((1, 1), (1, 1), (0, 0)), mode="wrap")


def _bf16_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV).to(torch.bfloat16)


def _pack(w, groups):
    """[co_total][ci][3][3] -> [groups][9][64][64] (group g holds co = 4c + g when groups = 4)."""
    out = np.zeros((groups, 9, 64, 64))
    for g in range(groups):
        co = np.arange(64) * 4 + g if groups == 4 else np.arange(64)
        out[g] = w[co].reshape(64, 64, 9).transpose(2, 0, 1)
    return out


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["prelu", "residual", "shuffle"])
@pytest.mark.parametrize("H,W", [(1024, 128), (16, 256)])
def test_tensor_core_conv_layer_matches_fp64(mg, mode, H, W):
    rng = np.random.default_rng(10 * mode + H)
    groups = 4 if mode == 2 else 1
    x = og.bf16_round(rng.standard_normal((H, W, 64)))
    w = og.bf16_round(rng.standard_normal((64 * groups, 64, 3, 3)) * np.sqrt(2.0 / 576))
    b = rng.standard_normal(64 * groups) * 0.1
    a = rng.uniform(0.05, 0.3, 64)
    skip = og.bf16_round(rng.standard_normal((H, W, 64)))
    xin = _bf16_dev(_pad(x))
    sk = _bf16_dev(_pad(skip))
    wp = _bf16_dev(_pack(w, groups))
    bias = torch.tensor(_pack_bias(b, groups), dtype=torch.float32, device=DEV)
    pre = torch.tensor(a, dtype=torch.float32, device=DEV)
    oh, ow = (2 * H, 2 * W) if mode == 2 else (H, W)
    out = torch.full((oh + 2, ow + 2, 64), float("nan"), dtype=torch.bfloat16, device=DEV)
    mg.op_sr_conv(mode, H, W, xin, sk if mode == 1 else None, wp, bias, pre if mode != 1 else None, out)
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().astype(np.float64)
    y = og.conv3x3(x.transpose(2, 0, 1), w, b)  # (64 * groups, H, W)
    if mode == 0:
        ref = og.prelu(y, a)
    elif mode == 1:
        ref = y + skip.transpose(2, 0, 1)
    else:
        ref = og.prelu(og.pixel_shuffle2(y), a)
    ref = ref.transpose(1, 2, 0)  # (oh, ow, 64)
    inner = got[1:-1, 1:-1]
    tol = 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max()
    bad = np.abs(inner - ref) > tol
    assert not bad.any(), (bad.sum(), np.abs(inner - ref).max())
    np.testing.assert_array_equal(got, _pad(inner))  # the halo holds the wrapped interior


def _pack_bias(b, groups):
    if groups == 1:
        return b
    return np.stack([b[np.arange(64) * 4 + g] for g in range(groups)])


def _small_weights(seed, gain=0.5, out_scale=1.0):
    w = random_weights(seed, gain=gain)
    w["out.w"] = w["out.w"] * out_scale
    w["out.b"] = w["out.b"] * out_scale
    return w


def test_generator_matches_bf16_oracle(mg):
    from paper_2403_07936_gb300 import sr
    nc = 128
    w = _small_weights(3)
    ctx = mg.Context(6, 2 * nc)
    ctx.load_weights(sr.pack_weights(w))
    ec = turbulent_source(nc, 16, 5) * 1e-3
    ect = torch.tensor(ec, dtype=torch.float32, device=DEV)
    out = torch.empty((2 * nc, 2 * nc), dtype=torch.float32, device=DEV)
    mg.op_sr_generator(ctx, ect, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    ec32 = ect.double().cpu().numpy()
    s = og.sr_scale(ec32)
    ref_bf16 = s * og.generator_forward(ec32 / s, w, emulate_bf16=True)
    ref_fp64 = s * og.generator_forward(ec32 / s, w)
    rel = np.linalg.norm(got - ref_bf16) / np.linalg.norm(ref_bf16)
    rel64 = np.linalg.norm(got - ref_fp64) / np.linalg.norm(ref_fp64)
    assert rel <= 1e-2, rel
    assert rel64 <= 3e-2, rel64


def test_sr_solve_with_zero_output_layer_equals_cubic(mg):
    """G = 0 (zero last layer): the SR prolongation is the cubic one, bit for bit."""
    from paper_2403_07936_gb300 import sr
    n = 256
    w = _small_weights(4, out_scale=0.0)
    f = turbulent_source(n, 32, 8)
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(6, n)
    ctx.load_weights(sr.pack_weights(w))
    ctx.set_options(inner_cycles=2)  # SR solves use a fixed count; the cubic one then uses it too
    a = torch.zeros_like(ft)
    b = torch.zeros_like(ft)
    ia = ctx.solve(ft, a, prolong="cubic")
    ib = ctx.solve(ft, b, prolong="sr")
    assert torch.equal(a, b) and ia["vcycles"] == ib["vcycles"]


@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_sr_solve_converges_to_oracle_solution(mg, graphs):
    from paper_2403_07936_gb300 import sr
    n = 512
    w = _small_weights(5, gain=0.5, out_scale=0.2)
    f = turbulent_source(n, 64, 9)
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(7, n)
    ctx.set_graph_execution(graphs)
    ctx.load_weights(sr.pack_weights(w))
    x = torch.zeros_like(ft)
    info = ctx.solve(ft, x, prolong="sr")
    assert info["rel_residual"] <= 1e-10 and info["prolong_used"] == 1
    xg = x.cpu().numpy()
    xe = omg.exact_solve_fft(f - f.mean())
    assert np.abs(xg - xe).max() <= 1e-9 * np.abs(xe).max()
    assert omg.relative_residual(f - f.mean(), xg, omg.grid_h(n)) <= 1e-10 + 2e-16 * 8 / omg.grid_h(n) ** 2


def test_sr_requires_weights_and_large_enough_grid(mg):
    n = 128
    ctx = mg.Context(5, n)
    ft = torch.tensor(turbulent_source(n, 16, 1), device=DEV)
    with pytest.raises(mg.MGError) as e:
        ctx.solve(ft, torch.zeros_like(ft), prolong="sr")
    assert e.value.status == 6  # MG_ERR_NO_WEIGHTS


TRAINED = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.dirname(
    __import__("os").path.abspath(__file__))), "paper_2403_07936_gb300", "weights", "sr_generator.mgsrw")


def _trained_blob(out_scale=1.0):
    from paper_2403_07936_gb300 import sr
    blob = open(TRAINED, "rb").read()
    if out_scale == 1.0:
        return blob
    w = sr.unpack_weights(blob)
    w["out.w"] = w["out.w"] * out_scale
    w["out.b"] = w["out.b"] * out_scale
    return sr.pack_weights(w)


def _policy_solve(mg, n, blob, graphs, n_gan=float("inf"), s_thres=0.0, prolong="sr", seed=21):
    f = turbulent_source(n, n // 8, seed)
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(int(np.log2(n // 8)) + 1, n)
    ctx.set_graph_execution(graphs)
    ctx.set_options(inner_cycles=2)  # the SR schedule, for cubic comparisons too
    ctx.load_weights(blob)
    ctx.set_prolong_policy(n_gan, s_thres)
    x = torch.zeros_like(ft)
    info = ctx.solve(ft, x, prolong=prolong)
    return f, x, info


def _assert_exact(f, x):
    xe = omg.exact_solve_fft(f - f.mean())
    assert np.abs(x.cpu().numpy() - xe).max() <= 1e-9 * np.abs(xe).max()


def test_trained_generator_needs_fewer_vcycles_than_cubic(mg):
    blob = _trained_blob()
    f, xc, ic = _policy_solve(mg, 512, blob, True, prolong="cubic")
    f, xs, isr = _policy_solve(mg, 512, blob, True)
    assert isr["sr_cycles"] == isr["vcycles"] and isr["sr_fallback"] == 0
    assert isr["vcycles"] < ic["vcycles"], (isr["vcycles"], ic["vcycles"])
    _assert_exact(f, xs)


@pytest.mark.parametrize("n_gan,s_thres", [(1.0, 0.0), (0.5, 0.0), (float("inf"), 1e-5), (1e-6, 0.0)],
                         ids=["alternate", "two-cubic-per-sr", "switch-at-1e-5", "cubic-only"])
def test_prolongation_policies(mg, n_gan, s_thres):
    blob = _trained_blob()
    f, xg, ig = _policy_solve(mg, 512, blob, True, n_gan, s_thres)
    _, xh, ih = _policy_solve(mg, 512, blob, False, n_gan, s_thres)
    assert torch.equal(xg, xh) and ig["vcycles"] == ih["vcycles"] and ig["sr_cycles"] == ih["sr_cycles"]
    assert ig["rel_residual"] <= 1e-10 and ig["sr_fallback"] == 0
    _assert_exact(f, xg)
    vc, nsr = ig["vcycles"], ig["sr_cycles"]
    if n_gan == 1.0:
        assert nsr == (vc + 1) // 2  # odd V-cycles use SR
    elif n_gan == 0.5:
        assert nsr == vc // 3  # every third V-cycle uses SR
    elif n_gan == 1e-6:
        _, xc, ic = _policy_solve(mg, 512, blob, True, prolong="cubic")
        assert nsr == 0 and ig["prolong_used"] == 0 and torch.equal(xg, xc)
    else:
        assert 0 < nsr < vc


@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_diverging_generator_falls_back_to_cubic(mg, graphs):
    """Weights scaled x100 make the SR correction useless: the first outer step
    does not halve the residual, SR is dropped and the solve still converges."""
    f, x, info = _policy_solve(mg, 512, _trained_blob(out_scale=100.0), graphs)
    assert info["sr_fallback"] == 1 and info["status"] == "MG_OK"
    assert info["sr_cycles"] == 2  # the first outer step's inner V-cycles
    assert info["rel_residual"] <= 1e-10
    _assert_exact(f, x)
