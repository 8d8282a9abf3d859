"""Batched solves of many right-hand sides of different sizes (GPU).

The batched graph runs the same tile kernels as a single solve, but its FP64
sums use a different block split, so results agree with the single solves to
rounding: the bound is the spec one, |x_batch - x_alone|_inf <=
1e-9 |x_alone|_inf, with each result also checked against the exact FFT
solution and for its own relative residual.
"""
import os

import numpy as np
import pytest

from oracle import multigrid as omg
from synthetic.sources import config_seed, default_kmax, turbulent_source

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _levels(n, coarsest=8):
    return int(np.log2(n // coarsest)) + 1


def _case(sizes, seed0):
    fs = [turbulent_source(n, default_kmax(n), config_seed(3, seed0 + i)) for i, n in enumerate(sizes)]
    return fs, [torch.tensor(f, device=DEV) for f in fs]


@pytest.mark.parametrize("sizes", [[256, 512, 256, 1024, 64, 512, 128],
                                   [256] * 6 + [512] * 3 + [1024]])
def test_batch_matches_single_solves_and_exact(mg, sizes):
    fs, fts = _case(sizes, 10 * len(sizes))
    ctxs = [mg.Context(_levels(n), n) for n in sizes]
    xs = [torch.zeros_like(ft) for ft in fts]
    infos = mg.solve_batched(ctxs, fts, xs, tol=1e-10)
    for f, ft, x, ctx, info in zip(fs, fts, xs, ctxs, infos):
        assert info["rel_residual"] <= 1e-10
        xa = torch.zeros_like(ft)
        ctx.solve(ft, xa, tol=1e-10)
        got, alone = x.cpu().numpy(), xa.cpu().numpy()
        assert np.abs(got - alone).max() <= 1e-9 * np.abs(alone).max()
        xe = omg.exact_solve_fft(f - f.mean())
        assert np.abs(got - xe).max() <= 1e-9 * np.abs(xe).max()
        h = omg.grid_h(f.shape[0])
        assert omg.relative_residual(f - f.mean(), got, h) <= 1e-10 + 2e-16 * 8 / h ** 2  # FP64 recomputation margin


def test_batch_graph_is_reused_and_handles_converged_members(mg):
    sizes = [256, 512, 256]
    fs, fts = _case(sizes, 77)
    ctxs = [mg.Context(_levels(n), n) for n in sizes]
    xs = [torch.zeros_like(ft) for ft in fts]
    mg.solve_batched(ctxs, fts, xs, tol=1e-10)
    # x[1] is now converged: it does no cycle, the others (reset) do
    xs[0].zero_()
    xs[2].zero_()
    infos = mg.solve_batched(ctxs, fts, xs, tol=1e-10)
    assert infos[1]["vcycles"] == 0 and infos[0]["vcycles"] > 0 and infos[2]["vcycles"] > 0
    for f, x in zip(fs, xs):
        xe = omg.exact_solve_fft(f - f.mean())
        assert np.abs(x.cpu().numpy() - xe).max() <= 1e-9 * np.abs(xe).max()


def test_batch_reports_nonfinite_member_and_solves_the_rest(mg):
    sizes = [256, 256]
    fs, fts = _case(sizes, 91)
    fts[1][5, 7] = float("inf")
    ctxs = [mg.Context(_levels(n), n) for n in sizes]
    xs = [torch.zeros_like(ft) for ft in fts]
    with pytest.raises(mg.MGError) as e:
        mg.solve_batched(ctxs, fts, xs, tol=1e-10)
    assert e.value.status == 8
    xe = omg.exact_solve_fft(fs[0] - fs[0].mean())
    assert np.abs(xs[0].cpu().numpy() - xe).max() <= 1e-9 * np.abs(xe).max()


def test_batch_falls_back_for_fp64_contexts(mg):
    sizes = [128, 256]
    fs, fts = _case(sizes, 55)
    ctxs = [mg.Context(_levels(n), n, precision="fp64") for n in sizes]
    xs = [torch.zeros_like(ft) for ft in fts]
    infos = mg.solve_batched(ctxs, fts, xs, tol=1e-10)
    for f, x, info in zip(fs, xs, infos):
        assert info["rel_residual"] <= 1e-10
        xe = omg.exact_solve_fft(f - f.mean())
        assert np.abs(x.cpu().numpy() - xe).max() <= 1e-9 * np.abs(xe).max()


def test_batch_of_the_full_mixed_size_workload(mg):
    """The batched workload itself: 256 right-hand sides, 128 at 256^2, 96 at
    512^2 and 32 at 1024^2 (67.1 M points), independent k^-5/3 sources (the
    benchmark's seeds), one batched graph.  Every member reports a relative
    residual <= 1e-10; every eighth member (16 + 12 + 4: all three sizes) is
    checked against the exact FFT solution to 1e-9."""
    sizes = [256] * 128 + [512] * 96 + [1024] * 32
    fs = [turbulent_source(n, n // 8, config_seed(3, i)) for i, n in enumerate(sizes)]
    fts = [torch.tensor(f, device=DEV) for f in fs]
    ctxs = [mg.Context(_levels(n), n) for n in sizes]
    xs = [torch.zeros_like(ft) for ft in fts]
    infos = mg.solve_batched(ctxs, fts, xs, tol=1e-10)
    assert all(i["rel_residual"] <= 1e-10 for i in infos)  # (a failing member raises)
    for k in range(0, len(sizes), 8):
        f = fs[k]
        xe = omg.exact_solve_fft(f - f.mean())
        got = xs[k].cpu().numpy()
        assert np.abs(got - xe).max() <= 1e-9 * np.abs(xe).max(), (k, sizes[k])
        assert abs(got.mean()) <= 1e-12 * np.abs(got).max()


TRAINED = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2403_07936_gb300",
                       "weights", "sr_generator.mgsrw")


@pytest.mark.parametrize("graphs", [True, False], ids=["single-graph", "single-hostloop"])
def test_sr_batch_matches_single_sr_solves_and_exact(mg, graphs):
    """The SR prolongation inside the batched graph (Algorithm 5 inside
    Algorithm 6 for every right-hand side): members of all three sizes of the
    batched workload (reduced counts) and one 128^2 member, whose 64^2 coarse
    grid the generator does not take, so it stays cubic.  Each member equals
    its own single SR solve (same V-cycle and SR-cycle counts, solution within
    1e-9; the generator kernels are the same, the FP64 sums use another block
    split) and the exact FFT solution to 1e-9."""
    blob = open(TRAINED, "rb").read()
    sizes = [256, 512, 256, 1024, 512, 256, 1024, 128]
    fs, fts = _case(sizes, 500)
    ctxs = []
    for n in sizes:
        c = mg.Context(_levels(n), n)
        c.load_weights(blob)
        c.set_options(inner_cycles=2)
        ctxs.append(c)
    xs = [torch.zeros_like(ft) for ft in fts]
    infos = mg.solve_batched(ctxs, fts, xs, tol=1e-10, prolong="sr")
    for n, f, ft, x, ctx, info in zip(sizes, fs, fts, xs, ctxs, infos):
        assert info["rel_residual"] <= 1e-10
        got = x.cpu().numpy()
        xe = omg.exact_solve_fft(f - f.mean())
        assert np.abs(got - xe).max() <= 1e-9 * np.abs(xe).max(), n
        if n == 128:
            assert info["sr_cycles"] == 0 and info["prolong_used"] == 0
            continue
        assert info["prolong_used"] == 1 and info["sr_cycles"] > 0
        ctx.set_graph_execution(graphs)
        xa = torch.zeros_like(ft)
        ia = ctx.solve(ft, xa, tol=1e-10, prolong="sr")
        assert (ia["vcycles"], ia["sr_cycles"], ia["sr_fallback"]) == \
            (info["vcycles"], info["sr_cycles"], info["sr_fallback"]), (n, ia, info)
        alone = xa.cpu().numpy()
        assert np.abs(got - alone).max() <= 1e-9 * np.abs(alone).max()


def test_sr_batch_falls_back_per_member(mg):
    """A generator whose output is scaled x100 makes the SR correction useless:
    every member drops SR after its first outer step (two SR V-cycles) and
    still converges to the exact solution; the cubic members are unaffected."""
    from paper_2403_07936_gb300 import sr
    w = sr.unpack_weights(open(TRAINED, "rb").read())
    w["out.w"] = w["out.w"] * 100.0
    w["out.b"] = w["out.b"] * 100.0
    blob = sr.pack_weights(w)
    sizes = [256, 512, 128]
    fs, fts = _case(sizes, 600)
    ctxs = []
    for n in sizes:
        c = mg.Context(_levels(n), n)
        c.load_weights(blob)
        c.set_options(inner_cycles=2)
        ctxs.append(c)
    xs = [torch.zeros_like(ft) for ft in fts]
    infos = mg.solve_batched(ctxs, fts, xs, tol=1e-10, prolong="sr")
    for n, f, x, info in zip(sizes, fs, xs, infos):
        assert info["rel_residual"] <= 1e-10
        xe = omg.exact_solve_fft(f - f.mean())
        assert np.abs(x.cpu().numpy() - xe).max() <= 1e-9 * np.abs(xe).max()
        if n == 128:
            assert info["sr_fallback"] == 0 and info["sr_cycles"] == 0
        else:
            assert info["sr_fallback"] == 1 and info["sr_cycles"] == 2
