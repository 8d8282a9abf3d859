"""TMA staging of the smoother's tiles (GPU).

With mg_set_tma_tiles(1) a single solve's FP32 down passes on 64-row tiles
(V(2, .), the default tile of the 1024^2 and 2048^2 levels) stage every
interior tile by tiled 2D TMA copies of x and b and split them into the red
and black arrays in shared memory; tiles whose halo wraps around the periodic
grid keep the 16-byte vector loads.  The arithmetic of every tile is the
same, so solves must agree bit for bit with the vector-load path, in a CUDA
graph and in the host loop, and still meet the solve bar against the exact
FFT solution.
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


@pytest.mark.parametrize("n", [1024, 2048])
@pytest.mark.parametrize("graphs", [True, False], ids=["graph", "hostloop"])
def test_tma_tiles_give_the_bits_of_vector_loads(mg, n, graphs):
    f = turbulent_source(n, default_kmax(n), config_seed(2, 40 + n // 1024))
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(_levels(n), n)
    ctx.set_graph_execution(graphs)
    mode = mg.get_tma_tiles()
    out = {}
    try:
        for on in (False, True):
            mg.set_tma_tiles(on)
            x = torch.zeros_like(ft)
            info = ctx.solve(ft, x, tol=1e-10)
            torch.cuda.synchronize()
            out[on] = (x.cpu().numpy(), info)
    finally:
        mg.set_tma_tiles(mode)
    (x0, i0), (x1, i1) = out[False], out[True]
    assert i0["vcycles"] == i1["vcycles"] and i0["outer_iters"] == i1["outer_iters"]
    assert np.array_equal(x0, x1)
    assert i1["rel_residual"] <= 1e-10
    xe = omg.exact_solve_fft(f - f.mean())
    assert np.abs(x1 - xe).max() <= 1e-9 * np.abs(xe).max()


def test_tma_tiles_switch(mg):
    mode = mg.get_tma_tiles()
    try:
        mg.set_tma_tiles(True)
        assert mg.get_tma_tiles()
        mg.set_tma_tiles(False)
        assert not mg.get_tma_tiles()
    finally:
        mg.set_tma_tiles(mode)
