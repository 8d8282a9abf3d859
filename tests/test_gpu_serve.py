"""Continuous-batching server (GPU).

Requests of mixed sizes join and leave the running batch between ticks.  Each
request runs the same batched kernels with its own reduction layout, and with
adaptive V-cycles a count chosen from its own residuals alone, so its result
does not depend on what else is in flight: a request served alone and the
same request served inside a mix of arrivals give identical bits, and with a
fixed count both equal a one-request batched solve.  Every result is also
checked against the exact FFT solution (|x - x_exact|_inf <= 1e-9
|x_exact|_inf) and for its own relative residual.
"""
import numpy as np
import pytest

from oracle import multigrid as omg
from synthetic.sources import config_seed, default_kmax, perturbed_source, turbulent_source

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GB = 1 << 30


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _src(n, i):
    return turbulent_source(n, default_kmax(n), config_seed(5, i))


def _drain(srv, max_ticks=500):
    out = []
    for _ in range(max_ticks):
        active, queued, _ = srv.tick()
        out += srv.poll()
        if active == 0 and queued == 0:
            return out
    raise AssertionError("server did not drain")


def _check_exact(f, x):
    xe = omg.exact_solve_fft(f - f.mean())
    assert np.abs(x - xe).max() <= 1e-9 * np.abs(xe).max()
    h = omg.grid_h(f.shape[0])
    assert omg.relative_residual(f - f.mean(), x, h) <= 1e-10 + 2e-16 * 8 / h ** 2  # FP64 recomputation margin


@pytest.mark.parametrize("inner", [0, 2, 5])  # adaptive; fixed V-cycles per outer step
def test_request_alone_equals_request_in_mix(mg, inner):
    f = _src(512, 0)
    ft = torch.tensor(f, device=DEV)
    alone = torch.zeros_like(ft)
    srv = mg.Server(8 * GB, inner_cycles=inner)
    srv.submit(ft, alone)
    res = _drain(srv)
    assert len(res) == 1 and res[0]["status"] == 0
    srv.close()

    others = [_src(n, 10 + i) for i, n in enumerate([256, 1024, 128, 512, 2048, 256])]
    ots = [torch.tensor(g, device=DEV) for g in others]
    oxs = [torch.zeros_like(t) for t in ots]
    mixed = torch.full_like(ft, float("nan"))
    srv = mg.Server(8 * GB, inner_cycles=inner)
    srv.submit(ots[0], oxs[0])
    srv.submit(ots[1], oxs[1])
    srv.tick()
    srv.submit(ots[2], oxs[2])
    srv.tick()
    rid = srv.submit(ft, mixed)  # joins a batch already two steps in
    srv.submit(ots[3], oxs[3])
    srv.tick()
    srv.submit(ots[4], oxs[4])
    srv.submit(ots[5], oxs[5])
    res = srv.poll() + _drain(srv)
    assert sorted(r["request_id"] for r in res) == list(range(7))
    assert all(r["status"] == 0 and r["rel_residual"] <= 1e-10 for r in res)
    assert torch.equal(alone, mixed)
    mine = [r for r in res if r["request_id"] == rid][0]
    assert mine["t_submit_ms"] <= mine["t_admit_ms"] <= mine["t_finish_ms"]
    _check_exact(f, mixed.cpu().numpy())
    for g, x in zip(others, oxs):
        _check_exact(g, x.cpu().numpy())

    if inner == 0:
        return
    # the same request as a one-member batched solve: the same kernels and sums
    ctx = mg.Context(7, 512)
    ctx.set_options(inner_cycles=inner)
    xb = torch.zeros_like(ft)
    mg.solve_batched([ctx], [ft], [xb], tol=1e-10)
    assert torch.equal(alone, xb)


def test_warm_start_stream_and_host_buffers(mg):
    n = 256
    f0 = _src(n, 40)
    fs = [f0]
    for k in range(3):
        fs.append(perturbed_source(fs[-1], config_seed(5, 100 + k)))
    srv = mg.Server(4 * GB)
    cycles = []
    for f in fs:
        fh = np.ascontiguousarray(f)
        xh = np.zeros_like(fh)
        srv.submit(fh, xh, stream_id=3)
        res = _drain(srv)
        assert len(res) == 1 and res[0]["status"] == 0 and res[0]["stream_id"] == 3
        cycles.append(res[0]["vcycles"])
        _check_exact(f, xh)
    # a 1% perturbation warm-started from the previous solution needs fewer cycles
    assert max(cycles[1:]) < cycles[0], cycles


def test_admission_respects_memory_budget(mg):
    n = 1024
    fs = [_src(n, 60 + i) for i in range(3)]
    fts = [torch.tensor(f, device=DEV) for f in fs]
    xs = [torch.zeros_like(t) for t in fts]
    # room for the server's tables and one 1024^2 hierarchy, not two
    srv = mg.Server(int(0.06 * GB))
    for t, x in zip(fts, xs):
        srv.submit(t, x)
    seen_active = []
    res = []
    for _ in range(200):
        a, q, _ = srv.tick()
        seen_active.append(a)
        res += srv.poll()
        if a == 0 and q == 0:
            break
    assert len(res) == 3 and max(seen_active) == 1
    for f, x in zip(fs, xs):
        _check_exact(f, x.cpu().numpy())
    with pytest.raises(mg.MGError) as e:
        srv.submit(torch.zeros((4096, 4096), dtype=torch.float64, device=DEV))
    assert e.value.status == 2  # MG_ERR_OOM: larger than the whole budget


def test_failures_retire_with_status_and_do_not_disturb_others(mg):
    n = 256
    good = _src(n, 80)
    bad = good.copy()
    bad[7, 9] = np.nan
    gt, bt = torch.tensor(good, device=DEV), torch.tensor(bad, device=DEV)
    gx, bx = torch.zeros_like(gt), torch.zeros_like(bt)
    srv = mg.Server(4 * GB)
    ig = srv.submit(gt, gx)
    ib = srv.submit(bt, bx)
    res = {r["request_id"]: r for r in _drain(srv)}
    assert res[ig]["status"] == 0 and res[ib]["status"] == 8  # MG_ERR_NONFINITE
    _check_exact(good, gx.cpu().numpy())
    srv.close()
    # a cycle cap below what the tolerance needs: MG_ERR_NOT_CONVERGED with the
    # best x so far (adaptive: 3 V-cycles, then the 1 left)
    srv = mg.Server(4 * GB, max_cycles=4)
    x = torch.zeros_like(gt)
    srv.submit(gt, x)
    (r,) = _drain(srv)
    assert r["status"] == 4 and r["vcycles"] == 4 and 0 < r["rel_residual"] < 1e-3


def test_constant_source_gives_zero(mg):
    n = 128
    f = torch.full((n, n), 3.0, dtype=torch.float64, device=DEV)
    x = torch.full_like(f, 5.0)
    srv = mg.Server(GB)
    srv.submit(f, x)
    (r,) = _drain(srv)
    assert r["status"] == 0 and r["vcycles"] == 0
    assert torch.count_nonzero(x) == 0
