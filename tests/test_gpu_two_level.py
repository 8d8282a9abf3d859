"""The paper's two-level x16 configuration (GPU): one coarse level 16 times
coarser, 20 red-black sweeps on the finest grid, 10 coarse sweeps, the coarse
correction interpolated back by 16 in one step with the periodic cubic
spline.  One cycle is compared with the oracle's two_level_cycle (FP32 inner
arithmetic against FP64: 1e-5 of the largest value); a full solve must reach
the relative residual (recomputed by the oracle) and lie within 1e-7 of the
exact FFT solution.  The SR variant interpolates by 16 in four stages, each
the cubic spline by 2 plus the generator's correction: with the generator's
output layer zeroed it is the cubic spline by 16 again; with the trained
generator the solve runs under the prolongation policy and its fallback.
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
    assert omg.relative_residual(fc, xg, omg.grid_h(n)) <= 1e-10 + 2e-16 * 8 / omg.grid_h(n) ** 2
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


TRAINED = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2403_07936_gb300",
                       "weights", "sr_generator.mgsrw")


def _blob(out_scale=1.0):
    from paper_2403_07936_gb300 import sr
    w = sr.unpack_weights(open(TRAINED, "rb").read())
    w["out.w"] = w["out.w"] * out_scale
    w["out.b"] = w["out.b"] * out_scale
    return sr.pack_weights(w)


def test_sr_x16_with_zero_generator_output_is_the_cubic_x16_cycle(mg):
    """G = 0: each stage is the cubic spline by 2, and four of them make the
    cubic spline by 16 (the spline through the coarse nodes is also the spline
    through its own values at the finer nodes; pinned in the oracle tests), so
    one SR cycle is the oracle's cubic two-level cycle (2048^2, coarse 128^2)."""
    n = 2048
    f = turbulent_source(n, default_kmax(n), config_seed(9, 7))
    ctx = mg.Context(9, n)
    ctx.load_weights(_blob(0.0))
    x = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    info = ctx.two_level_solve(torch.tensor(f, device=DEV), x, coarsen_log2=4, nu_smooth=4, coarse_sweeps=3,
                               max_cycles=1, prolong="sr", check=False)
    assert info["status"] == "MG_ERR_NOT_CONVERGED" and info["vcycles"] == 1 and info["sr_cycles"] == 1
    fc = f - f.mean()
    ref = omg.two_level_cycle(np.zeros((n, n)), fc, omg.grid_h(n), factor=16, nu=4, coarse_sweeps=3)
    ref -= ref.mean()
    got = x.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("n_gan", [float("inf"), 1.0], ids=["sr-every-cycle", "alternate"])
def test_sr_x16_solve_with_trained_generator(mg, n_gan):
    """The trained generator at every stage: cycles use SR as the policy says
    until an SR cycle fails to reduce the residual (then cubic to the end);
    the residual falls either way."""
    n = 2048
    f = turbulent_source(n, default_kmax(n), config_seed(9, 8))
    ft = torch.tensor(f, device=DEV)
    ctx = mg.Context(9, n)
    ctx.load_weights(_blob())
    ctx.set_prolong_policy(n_gan, 0.0)
    cyc = 30
    xs = torch.zeros_like(ft)
    isr = ctx.two_level_solve(ft, xs, max_cycles=cyc, prolong="sr", check=False)
    xc = torch.zeros_like(ft)
    icu = ctx.two_level_solve(ft, xc, max_cycles=cyc, prolong="cubic", check=False)
    assert isr["status"] in ("MG_OK", "MG_ERR_NOT_CONVERGED") and isr["vcycles"] == cyc
    assert icu["sr_cycles"] == 0 and icu["prolong_used"] == 0
    assert np.isfinite(isr["rel_residual"]) and isr["rel_residual"] < 0.5
    assert isr["prolong_used"] == 1 and isr["sr_cycles"] >= 1
    if not isr["sr_fallback"]:
        assert isr["sr_cycles"] == (cyc if n_gan == float("inf") else (cyc + 1) // 2)
    assert omg.relative_residual(f - f.mean(), xs.cpu().numpy(), omg.grid_h(n)) <= 1.5 * isr["rel_residual"]
    # a second SR solve on the same context reuses the stages' generator
    # buffers (and their tensor maps): the same bits
    xs2 = torch.zeros_like(ft)
    isr2 = ctx.two_level_solve(ft, xs2, max_cycles=cyc, prolong="sr", check=False)
    assert torch.equal(xs, xs2) and isr2["sr_cycles"] == isr["sr_cycles"]


def test_sr_x16_needs_weights_and_a_coarse_grid_of_128(mg):
    n = 1024
    ctx = mg.Context(8, n)
    f = torch.tensor(turbulent_source(n, 64, 3), device=DEV)
    with pytest.raises(mg.MGError) as e:
        ctx.two_level_solve(f, torch.zeros_like(f), prolong="sr")
    assert e.value.status == 6  # MG_ERR_NO_WEIGHTS
    ctx.load_weights(_blob())
    with pytest.raises(mg.MGError) as e:  # 1024 / 16 = 64 < 128
        ctx.two_level_solve(f, torch.zeros_like(f), prolong="sr")
    assert e.value.status == 1
    info = ctx.two_level_solve(f, torch.zeros_like(f), coarsen_log2=3, max_cycles=2, prolong="sr", check=False)
    assert info["sr_cycles"] >= 1  # 1024 / 8 = 128
