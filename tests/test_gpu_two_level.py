"""The paper's two-level x16 configuration (GPU): one coarse level 16 times
coarser, 20 red-black sweeps on the finest grid, 10 coarse sweeps, the coarse
correction interpolated back by 16 in one step with the periodic cubic
spline.  One cycle is compared with the oracle's two_level_cycle (FP32 inner
arithmetic against FP64: 1e-5 of the largest value); a full solve must reach
the relative residual (recomputed by the oracle) and lie within 1e-7 of the
exact FFT solution.
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


@pytest.mark.parametrize("nu,ncs", [(20, 10), (4, 3)])
def test_one_two_level_cycle_matches_oracle(mg, nu, ncs):
    n = 1024
    f = turbulent_source(n, default_kmax(n), config_seed(9, nu))
    ctx = mg.Context(8, n)
    x = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    info = ctx.two_level_solve(torch.tensor(f, device=DEV), x, coarsen_log2=4, nu_smooth=nu, coarse_sweeps=ncs,
                               max_cycles=1, check=False)
    assert info["status"] == "MG_ERR_NOT_CONVERGED" and info["vcycles"] == 1
    fc = f - f.mean()
    ref = omg.two_level_cycle(np.zeros((n, n)), fc, omg.grid_h(n), factor=16, nu=nu, coarse_sweeps=ncs)
    ref -= ref.mean()
    got = x.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def test_two_level_solve_converges_to_the_exact_solution(mg):
    n = 1024
    f = turbulent_source(n, default_kmax(n), config_seed(9, 100))
    ctx = mg.Context(8, n)
    x = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    info = ctx.two_level_solve(torch.tensor(f, device=DEV), x, tol=1e-10, max_cycles=400)
    assert info["status"] == "MG_OK" and info["rel_residual"] <= 1e-10
    fc = f - f.mean()
    xg = x.cpu().numpy()
    assert omg.relative_residual(fc, xg, omg.grid_h(n)) <= 1.5e-10
    # the error left at that residual is smooth (the weak coarse relaxation is
    # last to reduce the smooth modes, whose residual is small against their
    # size), so it is larger than after the multilevel V-cycle's 1e-9
    xe = omg.exact_solve_fft(fc)
    assert np.abs(xg - xe).max() <= 1e-7 * np.abs(xe).max()
    # the extreme coarsening needs many more cycles than the multilevel V-cycle
    xv = torch.zeros_like(x)
    assert ctx.solve(torch.tensor(f, device=DEV), xv)["vcycles"] < info["vcycles"]


def test_two_level_rejects_bad_arguments(mg):
    ctx = mg.Context(6, 256)
    f = torch.zeros((256, 256), dtype=torch.float64, device=DEV)
    x = torch.zeros_like(f)
    for kw in ({"coarsen_log2": 4}, {"coarsen_log2": 2, "coarse_sweeps": 0}, {"coarsen_log2": 2, "nu_smooth": 65}):
        with pytest.raises(mg.MGError) as e:
            ctx.two_level_solve(f, x, **kw)
        assert e.value.status == 1  # MG_ERR_INVALID_ARG
