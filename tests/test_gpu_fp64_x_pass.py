"""The FP64 V-cycle's prolongation pass along x, once per level (GPU).

With mg_set_fp64_separate_x_pass(1) (the default) an FP64 V-cycle refines
each level's coarse error along x once, over the whole grid
(k_refine_rows), and the up pass loads the refined rows instead of refining
them, with their halo, in every tile.  Each refined value is the same sum of
the same taps in the same order, so FP64 solves and single V-cycles must
agree bit for bit with the per-tile form, in a CUDA graph and in the host
loop, and the solves still meet the bar against the exact FFT solution.
"""
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


@pytest.mark.parametrize("n", [128, 512, 2048])
@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_separate_x_pass_gives_the_bits_of_per_tile_refinement(mg, n, graphs):
    f = turbulent_source(n, default_kmax(n), config_seed(2, 60 + n // 128))
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(_levels(n), n, precision="fp64")
    ctx.set_graph_execution(graphs)
    mode = mg.get_fp64_separate_x_pass()
    out = {}
    try:
        for on in (False, True):
            mg.set_fp64_separate_x_pass(on)
            x = torch.zeros_like(ft)
            info = ctx.solve(ft, x, tol=1e-10)
            torch.cuda.synchronize()
            out[on] = (x.cpu().numpy(), info)
    finally:
        mg.set_fp64_separate_x_pass(mode)
    (x0, i0), (x1, i1) = out[False], out[True]
    assert i0["vcycles"] == i1["vcycles"] and i0["rel_residual"] == i1["rel_residual"]
    assert np.array_equal(x0, x1)
    assert i1["rel_residual"] <= 1e-10
    xe = omg.exact_solve_fft(f - f.mean())
    assert np.abs(x1 - xe).max() <= 1e-9 * np.abs(xe).max()


def test_separate_x_pass_vcycle_matches_the_oracle(mg):
    """One FP64 V-cycle from x = 0 through mg_vcycle against the oracle's."""
    n = 256
    f = turbulent_source(n, default_kmax(n), config_seed(2, 66))
    f = f - f.mean()
    ctx = mg.Context(_levels(n), n, precision="fp64")
    assert mg.get_fp64_separate_x_pass()
    x = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    ctx.vcycle(torch.tensor(f, device=DEV), x)
    torch.cuda.synchronize()
    ref = omg.vcycle(np.zeros((n, n)), f, omg.grid_h(n), nu1=2, nu2=2, coarsest=8)
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


def test_separate_x_pass_switch(mg):
    mode = mg.get_fp64_separate_x_pass()
    try:
        mg.set_fp64_separate_x_pass(False)
        assert not mg.get_fp64_separate_x_pass()
        mg.set_fp64_separate_x_pass(True)
        assert mg.get_fp64_separate_x_pass()
        assert mg.load().mg_set_fp64_separate_x_pass(2) == 1  # MG_ERR_INVALID_ARG
    finally:
        mg.set_fp64_separate_x_pass(mode)
