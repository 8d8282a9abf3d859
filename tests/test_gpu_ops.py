"""Operator-level parity of the CUDA kernels against the oracle (GPU).

Each C-ABI operator entry point runs the production kernel on one grid; the
oracle runs the same step in FP64 with mesh width 1, which is exactly the
scaled formulation b = h^2 * rhs that the kernels use.

Tolerances: FP64 kernels agree with the oracle to rounding (the smoother
performs the same operations in the same order); the FP32 kernels are
compared with the FP64 oracle run on the same float-rounded inputs, and a few
sweeps of a contractive smoother keep the float error near a few ulp of the
largest value (bound 2e-6 relative to max|x|).
"""
import numpy as np
import pytest

from oracle import multigrid as omg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = {torch.float64: 1e-13, torch.float32: 2e-6}


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2403_07936_gb300 import mg as m
    return m


def _rand(n, seed, zero_mean=False):
    a = np.random.default_rng(seed).standard_normal((n, n))
    return a - a.mean() if zero_mean else a


def _as(a, dt):
    """Round to the test dtype and return (device tensor, float64 copy of the rounded values)."""
    t = torch.tensor(a, dtype=dt, device=DEV)
    return t, t.double().cpu().numpy()


def _relerr(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [64, 128, 256, 2048])
@pytest.mark.parametrize("nu,zero", [(0, False), (1, False), (2, False), (2, True), (3, False), (4, True)])
def test_down_matches_oracle(mg, dt, n, nu, zero):
    x, x64 = _as(_rand(n, 1), dt)
    b, b64 = _as(_rand(n, 2, zero_mean=True), dt)
    bc = torch.empty((n // 2, n // 2), dtype=dt, device=DEV)
    xo = torch.full_like(x, float("nan"))
    mg.op_down(x, xo, b, bc, nu=nu, zero_init=zero)
    torch.cuda.synchronize()
    xr = np.zeros_like(x64) if zero else x64.copy()
    omg.rbgs(xr, b64, 1.0, nu)
    bcr = 4.0 * omg.restrict_fw(omg.residual(b64, xr, 1.0))
    assert _relerr(xo.double().cpu().numpy(), xr) <= TOL[dt]
    np.testing.assert_array_equal(x.double().cpu().numpy(), x64)  # input untouched
    assert _relerr(bc.double().cpu().numpy(), bcr) <= 4 * TOL[dt]


def test_down_fp64_smoother_is_bit_exact(mg):
    n = 128
    x, x64 = _as(_rand(n, 3), torch.float64)
    b, b64 = _as(_rand(n, 4, zero_mean=True), torch.float64)
    bc = torch.empty((n // 2, n // 2), dtype=torch.float64, device=DEV)
    xo = torch.empty_like(x)
    mg.op_down(x, xo, b, bc, nu=2)
    torch.cuda.synchronize()
    xr = x64.copy()
    omg.rbgs(xr, b64, 1.0, 2)
    np.testing.assert_array_equal(xo.cpu().numpy(), xr)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [64, 128, 512, 2048])
@pytest.mark.parametrize("nu", [0, 1, 2, 4])
def test_up_matches_oracle(mg, dt, n, nu):
    x, x64 = _as(_rand(n, 5), dt)
    b, b64 = _as(_rand(n, 6, zero_mean=True), dt)
    ec, ec64 = _as(_rand(n // 2, 7), dt)
    xo = torch.empty_like(x)
    mg.op_up(x, xo, b, ec, nu=nu)
    torch.cuda.synchronize()
    xr = x64 + omg.prolong_cubic(ec64)
    omg.rbgs(xr, b64, 1.0, nu)
    assert _relerr(xo.double().cpu().numpy(), xr) <= TOL[dt]


def test_up_prolongation_of_constant_and_smooth_mode(mg):
    """P 1 = 1, and a smooth mode sampled on the coarse grid is interpolated
    within the cubic-spline bound (5/384) H^4 max|d^4 u| per axis."""
    n = 256
    x = torch.zeros((n, n), dtype=torch.float64, device=DEV)
    xo = torch.empty_like(x)
    ec = torch.full((n // 2, n // 2), 3.0, dtype=torch.float64, device=DEV)
    mg.op_up(x, xo, x.clone(), ec, nu=0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(xo.cpu().numpy(), 3.0, atol=1e-13)
    j = np.arange(n) * 2 * np.pi / n
    fine = np.sin(2 * j)[:, None] * np.cos(3 * j)[None, :]
    ec = torch.tensor(np.ascontiguousarray(fine[0::2, 0::2]), device=DEV)
    mg.op_up(x, xo, x.clone(), ec, nu=0)
    torch.cuda.synchronize()
    H = 2 * np.pi / (n // 2)
    bound = 5.0 / 384.0 * H ** 4 * (2 ** 4 + 3 ** 4)
    err = np.abs(xo.cpu().numpy() - fine).max()
    assert 0 < err <= bound


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,coarsest", [(8, 8), (8, 4), (16, 8), (32, 8), (64, 8), (64, 4), (64, 16)])
@pytest.mark.parametrize("nu1,nu2,zero", [(2, 2, True), (1, 1, False), (0, 3, False), (4, 0, True)])
def test_bottom_vcycle_matches_oracle(mg, dt, n, coarsest, nu1, nu2, zero):
    x, x64 = _as(_rand(n, 8), dt)
    b, b64 = _as(_rand(n, 9, zero_mean=True), dt)
    mg.op_vcycle(x, b, coarsest=coarsest, nu1=nu1, nu2=nu2, zero_init=zero)
    torch.cuda.synchronize()
    x0 = np.zeros_like(x64) if zero else x64
    xr = omg.vcycle(x0, b64, 1.0, nu1, nu2, coarsest=coarsest)
    tol = 1e-12 if dt == torch.float64 else 2e-5
    assert _relerr(x.double().cpu().numpy(), xr) <= tol


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("coarsest", [8, 16])
def test_bottom_vcycle_unaligned_buffers_match_aligned(mg, dt, coarsest):
    """x and b that start off a 16-byte boundary are staged (and written back)
    element by element instead of by 16-byte vector loads; the cycle's
    arithmetic is the same, so the result is bit-identical."""
    n = 64
    x, _ = _as(_rand(n, 12), dt)
    b, _ = _as(_rand(n, 13, zero_mean=True), dt)
    xb = torch.zeros(n * n + 1, dtype=dt, device=DEV)
    bb = torch.zeros(n * n + 1, dtype=dt, device=DEV)
    xu, bu = xb[1:].view(n, n), bb[1:].view(n, n)
    xu.copy_(x)
    bu.copy_(b)
    assert xu.data_ptr() % 16 != 0 and bu.data_ptr() % 16 != 0 and x.data_ptr() % 16 == 0
    mg.op_vcycle(x, b, coarsest=coarsest, nu1=2, nu2=2)
    mg.op_vcycle(xu, bu, coarsest=coarsest, nu1=2, nu2=2)
    torch.cuda.synchronize()
    assert torch.equal(x, xu) and torch.isfinite(x).all()


RED_BLOCKS, RED_THREADS = 304, 256  # grid of the FP64 outer kernels


def test_outer_residual_matches_oracle(mg):
    n = 256
    h = omg.grid_h(n)
    f = _rand(n, 10) + 0.3
    x = _rand(n, 11)
    mu = f.mean()
    ft = torch.tensor(f, device=DEV)
    xt = torch.tensor(x, device=DEV)
    s32 = torch.empty((n, n), dtype=torch.float32, device=DEV)
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    mg.op_outer_residual(ft, xt, mu, s32, out)
    torch.cuda.synchronize()
    s_ref = h * h * omg.residual(f - mu, x, h)
    np.testing.assert_allclose(s32.double().cpu().numpy(), s_ref, rtol=1e-6,
                               atol=1e-6 * np.abs(s_ref).max())
    o = out.cpu().numpy()
    # the norm sums squares of float-rounded residuals, FP32 within a thread:
    # 2^-23 from the rounding plus 2^-24 per term of the longest thread sum
    terms = -(-(n * n) // (RED_BLOCKS * RED_THREADS))
    assert abs(o[0] - np.sum(s_ref ** 2)) <= (2.0 ** -23 + terms * 2.0 ** -24) * np.sum(s_ref ** 2)
    assert abs(o[1] - np.sum((f - mu) ** 2)) <= 1e-12 * np.sum((f - mu) ** 2)


def _exact_residual_inputs(case, n):
    rng = np.random.default_rng({"wide": 21, "cancelling": 22, "subnormal": 23}[case])
    h2 = omg.grid_h(n) ** 2
    if case == "wide":  # operands spread over 2^-30 .. 2^30, both signs
        x = rng.choice([-1.0, 1.0], (n, n)) * 2.0 ** rng.uniform(-30, 30, (n, n))
        f = rng.standard_normal((n, n)) * 2.0 ** rng.uniform(-10, 40, (n, n))
    elif case == "cancelling":  # b = 4x - sum to binary64 rounding: the residual is the rounding
        j = np.arange(n) * omg.grid_h(n)
        x = 1e6 * np.sin(j)[:, None] * np.cos(2 * j)[None, :] + rng.uniform(-1e-3, 1e-3, (n, n))
        f = (4.0 * x - omg.neighbour_sum(x)) / h2
    else:  # residuals in binary32's subnormal range
        x = rng.standard_normal((n, n)) * 1e-39
        f = rng.standard_normal((n, n)) * 1e-40 / h2
    return f, x, h2 * f  # b = h^2 (f - mu) with mu = 0, as the kernel forms it


def _task_max_operand(b, x, rows=8, cols=32):
    """Largest operand magnitude, max(4|x|, |b|), over each point's residual task:
    the task-tiled kernel's tiling of 32 columns x 8 rows, with the x rows just
    above and below it and the x columns just left and right of it."""
    n = x.shape[0]
    m = np.empty((n, n))
    for r0 in range(0, n, rows):
        for c0 in range(0, n, cols):
            rr = np.arange(r0 - 1, r0 + rows + 1) % n
            xs = np.abs(x[np.ix_(rr, np.arange(c0, c0 + cols))]).max()
            halo = np.abs(x[np.ix_(np.arange(r0, r0 + rows), [(c0 - 1) % n, (c0 + cols) % n])]).max()
            bs = np.abs(b[r0:r0 + rows, c0:c0 + cols]).max()
            m[r0:r0 + rows, c0:c0 + cols] = max(4 * xs, 4 * halo, bs)
    return m


@pytest.mark.parametrize("case", ["wide", "cancelling", "subnormal"])
def test_outer_residual_is_exact_before_its_float_rounding(mg, case):
    """The outer residual sums its binary64 operands exactly, as 64-bit integers
    aligned to the largest exponent of the point's task (32 columns x 8 rows),
    and rounds once to float: within 10 * 2^-59 of the task's largest operand,
    plus half a float ulp, of the exact rational residual.  In the cancelling
    case binary64 evaluation itself misses that bound."""
    from fractions import Fraction
    n = 32
    f, x, b = _exact_residual_inputs(case, n)
    s32 = torch.empty((n, n), dtype=torch.float32, device=DEV)
    out = torch.zeros(2, dtype=torch.float64, device=DEV)
    mg.op_outer_residual(torch.tensor(f, device=DEV), torch.tensor(x, device=DEV), 0.0, s32, out)
    torch.cuda.synchronize()
    got = s32.cpu().numpy()
    ex = omg.scaled_residual_exact(b, x)
    tol = 10 * 2.0 ** -59 * _task_max_operand(b, x)
    half_ulp = np.abs(np.spacing(got)).astype(np.float64) / 2
    r64 = omg.residual(b, x, 1.0)
    fp64_ok = True
    for i in range(n):
        for j in range(n):
            bound = Fraction(float(tol[i, j])) + Fraction(float(half_ulp[i, j]))
            err = abs(Fraction(float(got[i, j])) - ex[i][j])
            assert err <= bound, (i, j, got[i, j], float(ex[i][j]))
            fp64_ok &= abs(Fraction(float(np.float32(r64[i, j]))) - ex[i][j]) <= bound
    if case == "cancelling":
        assert not fp64_ok
    if case == "subnormal":
        assert np.any((got != 0) & (np.abs(got) < np.finfo(np.float32).tiny))


def _conversion_inputs_f64():
    rng = np.random.default_rng(5)
    mant = rng.uniform(1.0, 2.0, 200000) * rng.choice([-1.0, 1.0], 200000)
    v = np.ldexp(mant, rng.integers(-160, 140, 200000))
    f = rng.standard_normal(50000).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + g.astype(np.float64)) / 2  # exact ties
    eps = np.abs(mid) * 2.0 ** -45
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax * (1 + 2.0 ** -25),
                        fmax * (1 + 2.0 ** -24), tiny, tiny * (1 - 2.0 ** -30), tiny / 2, 2.0 ** -149,
                        2.0 ** -150, 5e-324, 1e308, 1.0, -1.0, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24])
    return np.concatenate([v, mid, mid + eps, mid - eps, special])


@pytest.mark.parametrize("direction", ["f64_to_f32", "f32_to_f64"])
def test_integer_pipe_conversions_match_hardware_bit_for_bit(mg, direction):
    torch = pytest.importorskip("torch")
    if direction == "f64_to_f32":
        src = torch.tensor(_conversion_inputs_f64(), dtype=torch.float64, device="cuda:0")
        out = torch.empty(src.shape, dtype=torch.float32, device="cuda:0")
        ref = src.to(torch.float32)
    else:
        rng = np.random.default_rng(6)
        bits = rng.integers(0, 2 ** 32, 300000, dtype=np.uint64).astype(np.uint32)
        src = torch.tensor(bits.view(np.float32), device="cuda:0")
        out = torch.empty(src.shape, dtype=torch.float64, device="cuda:0")
        ref = src.to(torch.float64)
    mg.op_convert(src, out)
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(out), nan)
    ib = torch.int32 if out.dtype == torch.float32 else torch.int64
    assert torch.equal(out[~nan].view(ib), ref[~nan].view(ib))
