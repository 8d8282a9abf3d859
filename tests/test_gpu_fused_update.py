"""The outer step's FP64 update fused with the next outer residual (GPU).

With mg_set_fused_update(1) (the default) a mixed solve applies x += e and
forms the next residual r = f - A x in one launch that writes x + e into the
other buffer of a pair (the caller's x and a context buffer, alternating each
outer step); the solve's projection reads whichever buffer holds the last
iterate and writes the caller's x.  Each stored value and each residual is the
arithmetic of the separate update and residual launches, so solves must agree
bit for bit with the unfused form (x, V-cycles, outer steps, relative
residual), in a CUDA graph and in the host loop, after odd and even numbers of
outer steps, on device and host buffers, when the solve stops unconverged, and
with the SR prolongation policy; the reported update norm is the same sum in
another order.  The fused solves still meet the solve bar against the exact
FFT solution.
"""
import os

import numpy as np
import pytest

from oracle import multigrid as omg
from synthetic.sources import config_seed, default_kmax, turbulent_source

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TRAINED = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2403_07936_gb300",
                       "weights", "sr_generator.mgsrw")


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _levels(n, coarsest=8):
    return int(np.log2(n // coarsest)) + 1


def _both(mg, ctx, f, x0, **kw):
    """Solve (f, x0) with the fused and the unfused outer step; results per mode."""
    mode = mg.get_fused_update()
    out = {}
    try:
        for on in (False, True):
            mg.set_fused_update(on)
            x = x0.clone() if x0.is_cuda else x0.clone().pin_memory()
            info = ctx.solve(f, x, **kw)
            if x.is_cuda:
                torch.cuda.synchronize()
            out[on] = (x.cpu().numpy(), info)
    finally:
        mg.set_fused_update(mode)
    return out


def _assert_same(out):
    (x0, i0), (x1, i1) = out[False], out[True]
    for k in ("vcycles", "outer_iters", "rel_residual", "status"):
        assert i0[k] == i1[k], (k, i0[k], i1[k])
    assert np.array_equal(x0, x1)
    assert i1["update_norm"] == pytest.approx(i0["update_norm"], rel=1e-12, abs=0.0)


@pytest.mark.parametrize("n", [32, 256, 2048])
@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
@pytest.mark.parametrize("tol", [1e-10, 1e-6, 1e-3])
def test_fused_update_gives_the_bits_of_separate_launches(mg, n, graphs, tol):
    f = turbulent_source(n, default_kmax(n), config_seed(2, 80 + n // 32))
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(_levels(n), n)
    ctx.set_graph_execution(graphs)
    out = _both(mg, ctx, ft, torch.zeros_like(ft), tol=tol)
    _assert_same(out)
    x1, i1 = out[True]
    assert i1["outer_iters"] >= 1 and i1["rel_residual"] <= tol
    if tol == 1e-10:
        xe = omg.exact_solve_fft(f - f.mean())
        assert np.abs(x1 - xe).max() <= 1e-9 * np.abs(xe).max()


def test_fused_update_covers_odd_and_even_outer_step_counts(mg):
    """The parametrised solves above must take both parities of outer steps,
    so that the last iterate is found in either buffer of the pair."""
    n = 256
    f = turbulent_source(n, default_kmax(n), config_seed(2, 80 + n // 32))
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(_levels(n), n)
    seen = set()
    for tol in (1e-10, 1e-6, 1e-3):
        out = _both(mg, ctx, ft, torch.zeros_like(ft), tol=tol)
        _assert_same(out)
        seen.add(out[True][1]["outer_iters"] % 2)
    assert seen == {0, 1}


@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_fused_update_from_a_nonzero_guess_and_host_buffers(mg, graphs):
    n = 512
    rng = np.random.default_rng(5)
    f = turbulent_source(n, default_kmax(n), config_seed(2, 91))
    x0 = rng.standard_normal((n, n)) * 1e-3
    ctx = mg.Context(_levels(n), n)
    ctx.set_graph_execution(graphs)
    dev = _both(mg, ctx, torch.tensor(f, device=DEV), torch.tensor(x0, device=DEV), tol=1e-10)
    _assert_same(dev)
    host = _both(mg, ctx, torch.tensor(f).pin_memory(), torch.tensor(x0), tol=1e-10)
    _assert_same(host)
    assert np.array_equal(host[True][0], dev[True][0])


@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_fused_update_when_the_solve_stops_unconverged(mg, graphs):
    n = 256
    f = turbulent_source(n, default_kmax(n), config_seed(2, 93))
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(_levels(n), n)
    ctx.set_graph_execution(graphs)
    # the adaptive rule takes 3 V-cycles in the first outer step and at most
    # the cycles left after it: a cap of 2 stops after 1 outer step, 4 after 2
    for cap, steps in ((2, 1), (4, 2)):
        ctx.set_options(max_cycles=cap)
        out = _both(mg, ctx, ft, torch.zeros_like(ft), tol=1e-14, check=False)
        assert out[True][1]["status"] == "MG_ERR_NOT_CONVERGED"
        assert out[True][1]["outer_iters"] == steps
        _assert_same(out)
        assert abs(out[True][0].mean()) <= 1e-12 * np.abs(out[True][0]).max()


@pytest.mark.skipif(not os.path.exists(TRAINED), reason="trained generator weights not present")
@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_fused_update_with_the_sr_policy(mg, graphs):
    n = 256
    f = turbulent_source(n, n // 8, 21)
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(_levels(n), n)
    ctx.set_graph_execution(graphs)
    ctx.set_options(inner_cycles=2)
    ctx.load_weights(open(TRAINED, "rb").read())
    ctx.set_prolong_policy(1.0, 0.0)  # SR and cubic V-cycles alternate
    out = _both(mg, ctx, ft, torch.zeros_like(ft), tol=1e-10, prolong="sr")
    _assert_same(out)
    assert out[True][1]["sr_cycles"] >= 1


def test_fused_update_switch(mg):
    mode = mg.get_fused_update()
    try:
        mg.set_fused_update(False)
        assert not mg.get_fused_update()
        mg.set_fused_update(True)
        assert mg.get_fused_update()
    finally:
        mg.set_fused_update(mode)


@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
@pytest.mark.parametrize("fused", [True, False], ids=["fused", "separate"])
@pytest.mark.parametrize("host", [False, True], ids=["device", "host"])
def test_cold_start_never_reads_x(mg, graphs, fused, host):
    """mg_set_zero_guess: with the fused outer step the first residual and the
    first update take x = 0 without reading x (x holds NaN here, which any read
    would carry into the result); the bits are those of a solve from zeros."""
    n = 256
    f = turbulent_source(n, default_kmax(n), config_seed(2, 95))
    ctx = mg.Context(_levels(n), n)
    ctx.set_graph_execution(graphs)
    ft = torch.tensor(f, device=DEV)
    x0 = torch.zeros_like(ft)
    ref = ctx.solve(ft, x0, tol=1e-10)
    torch.cuda.synchronize()
    mode = mg.get_fused_update()
    try:
        mg.set_fused_update(fused)
        ctx.set_zero_guess(True)
        for tol, expect in ((1e-10, None), (2.0, "zeros")):  # tol >= 1: no outer step runs
            xg = torch.full((n, n), float("nan"), dtype=torch.float64)
            if host:
                fi, xg = torch.tensor(f).pin_memory(), xg.pin_memory()
            else:
                fi, xg = ft, xg.to(DEV)
            info = ctx.solve(fi, xg, tol=tol)
            torch.cuda.synchronize()
            got = xg.cpu().numpy()
            if expect == "zeros":
                assert info["outer_iters"] == 0 and np.array_equal(got, np.zeros((n, n)))
            else:
                assert info["vcycles"] == ref["vcycles"] and info["rel_residual"] == ref["rel_residual"]
                assert np.array_equal(got, x0.cpu().numpy())
    finally:
        ctx.set_zero_guess(False)
        mg.set_fused_update(mode)


def test_batched_fused_update_gives_the_bits_of_separate_launches(mg):
    """The batched graph's fused outer step: each member alternates its own
    iterate pair by its own outer-step count (members here end after
    different numbers of outer steps, one warm-started near its solution), and
    the projection reads each member's last buffer; the bits are those of the
    separate update and residual launches."""
    sizes = [256, 512, 64, 1024, 256]
    fs = [turbulent_source(n, default_kmax(n), config_seed(3, 200 + i)) for i, n in enumerate(sizes)]
    fts = [torch.tensor(f, device=DEV) for f in fs]
    warm = {}
    for i, tol in ((1, 1e-11), (4, 1e-6)):  # converged (no outer step), and part way
        ci = mg.Context(_levels(sizes[i]), sizes[i])
        w = torch.zeros_like(fts[i])
        ci.solve(fts[i], w, tol=tol)
        warm[i] = w
    mode = mg.get_fused_update()
    out = {}
    try:
        for on in (False, True):
            mg.set_fused_update(on)
            ctxs = [mg.Context(_levels(n), n) for n in sizes]
            xs = [warm[i].clone() if i in warm else torch.zeros_like(ft) for i, ft in enumerate(fts)]
            infos = mg.solve_batched(ctxs, fts, xs, tol=1e-10)
            torch.cuda.synchronize()
            out[on] = ([x.cpu().numpy() for x in xs], infos)
    finally:
        mg.set_fused_update(mode)
    (x0, i0), (x1, i1) = out[False], out[True]
    for k in range(len(sizes)):
        for key in ("vcycles", "outer_iters", "rel_residual"):
            assert i0[k][key] == i1[k][key], (k, key)
        assert np.array_equal(x0[k], x1[k]), k
        xe = omg.exact_solve_fft(fs[k] - fs[k].mean())
        assert np.abs(x1[k] - xe).max() <= 1e-9 * np.abs(xe).max()
    assert len({i["outer_iters"] % 2 for i in i1}) == 2  # both buffers of a pair hold a result
