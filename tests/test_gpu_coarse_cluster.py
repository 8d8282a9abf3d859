"""The coarse tail of a V-cycle as one thread-block-cluster launch (GPU).

With mg_set_coarse_cluster(1) a single solve runs the 128^2 level's down
pass, the bottom V-cycle (64^2 down to the coarsest grid and back) and the
128^2 level's up pass as one launch of an 8-CTA cluster whose phases are
ordered by the cluster barrier.  Every point's arithmetic is that of the
separate k_down, k_bottom and k_up launches, so solves must agree bit for bit
with the three-launch form, in a CUDA graph and in the host loop, for both
coarsest grids the bottom solve takes, and still meet the solve bar against
the exact FFT solution.
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


@pytest.mark.parametrize("n,coarsest", [(256, 8), (512, 16), (2048, 8), (128, 8)])
@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_cluster_tail_gives_the_bits_of_three_launches(mg, n, coarsest, graphs):
    f = turbulent_source(n, default_kmax(n), config_seed(2, 70 + n // 128))
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(int(np.log2(n // coarsest)) + 1, n)
    ctx.set_graph_execution(graphs)
    mode = mg.get_coarse_cluster()
    out = {}
    try:
        for on in (False, True):
            mg.set_coarse_cluster(on)
            x = torch.zeros_like(ft)
            info = ctx.solve(ft, x, tol=1e-10)
            torch.cuda.synchronize()
            out[on] = (x.cpu().numpy(), info)
    finally:
        mg.set_coarse_cluster(mode)
    (x0, i0), (x1, i1) = out[False], out[True]
    assert i0["vcycles"] == i1["vcycles"] and i0["outer_iters"] == i1["outer_iters"]
    assert np.array_equal(x0, x1)
    assert i1["rel_residual"] <= 1e-10
    xe = omg.exact_solve_fft(f - f.mean())
    assert np.abs(x1 - xe).max() <= 1e-9 * np.abs(xe).max()


def test_cluster_vcycle_matches_the_oracle_vcycle(mg):
    """One FP32 V-cycle of a 256^2 context through mg_vcycle equals the
    oracle's FP64 V-cycle to FP32 accuracy with the cluster tail on."""
    from synthetic.sources import turbulent_source as ts
    n = 256
    f = ts(n, default_kmax(n), config_seed(2, 99))
    f = f - f.mean()
    ctx = mg.Context(6, n)
    mode = mg.get_coarse_cluster()
    try:
        mg.set_coarse_cluster(True)
        x = torch.zeros((n, n), dtype=torch.float64, device=DEV)
        ctx.vcycle(torch.tensor(f, device=DEV), x)
        torch.cuda.synchronize()
    finally:
        mg.set_coarse_cluster(mode)
    ref = omg.vcycle(np.zeros((n, n)), f, omg.grid_h(n), nu1=2, nu2=2, coarsest=8)
    got = x.cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


def test_coarse_cluster_switch(mg):
    mode = mg.get_coarse_cluster()
    try:
        mg.set_coarse_cluster(False)
        assert not mg.get_coarse_cluster()
        mg.set_coarse_cluster(True)
        assert mg.get_coarse_cluster()
    finally:
        mg.set_coarse_cluster(mode)
