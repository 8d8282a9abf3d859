"""Plain FP64 CPU oracle of the periodic multigrid V-cycle.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
definition the CUDA path is checked against.  Only the tests, the smoke check
and the benchmark's CPU-baseline leg may import it; the product library never
does, and this module imports nothing from the product package.

Problem (Sec. 2.2, Eq. poissoneq; Sec. 3.2, Eq. poisson_ns).  The paper writes
the pressure-Poisson equation as Lap p = f with biperiodic velocity data and
leaves the boundary conditions unstated.  The reading used throughout:

* vertex grid x_j = j h, h = 2 pi / n, j = 0..n-1, periodic in both axes;
* A = -Lap_h, the 5-point stencil (A x)_ij = (4 x_ij - x_i+1,j - x_i-1,j
  - x_i,j+1 - x_i,j-1) / h^2 (sign flipped so that A is positive semi-definite);
* A is singular (constants), so the answer is the unique zero-mean solution
  x* = A^+ f of a zero-mean source.

Multigrid (Sec. 2.2, Fig. 1a; Appendix A, Algorithm 6), with these readings:

* smoother: Gauss-Seidel in red-black ordering (Sec. 2.2 names red-black
  ordering), red = (i + j) even first, then black; nu1 sweeps before and nu2
  after the coarse-grid correction (the paper shows pre-relaxation only and
  calls its count N_iter, which is garbled; V(2,2) is used here);
* residual r = f - A x (Algorithm 6);
* restriction: full weighting (the paper's example is injection of black
  points, Sec. 2.2; full weighting is the standard choice adopted here);
* coarse operator: the same 5-point stencil re-discretised at 2h;
* coarsest grid: exact solve (the paper relaxes 10 times, Algorithm 6);
* prolongation: periodic tensor-product cubic interpolating spline (the paper
  uses SciPy's bivariate spline, Sec. 2.2), added to the finer error;
* stopping: relative residual ||f - A x||_2 / ||f||_2 <= tol (the paper stops
  on |p_i - p_{i+1}| <= 1e-10, Sec. 4.2; the update norm is also returned).

Functions whose result has a closed form are pinned in tests/test_oracle_*.py
against that form, against dense brute force and against library routines
(numpy.linalg, scipy.interpolate.CubicSpline).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def grid_h(n: int) -> float:
    """Mesh width of the n x n periodic vertex grid on [0, 2 pi)."""
    return TWO_PI / n


# ---------------------------------------------------------------------------
# Operator, residual (Sec. 2.2 Eq. poissoneq; Algorithm 6 residual step)
# ---------------------------------------------------------------------------

def neighbour_sum(x: np.ndarray) -> np.ndarray:
    """Sum of the four periodic neighbours of every point."""
    return (np.roll(x, 1, axis=0) + np.roll(x, -1, axis=0)
            + np.roll(x, 1, axis=1) + np.roll(x, -1, axis=1))


def apply_A(x: np.ndarray, h: float) -> np.ndarray:
    """(A x)_ij = (4 x_ij - sum of 4 neighbours) / h^2, A = -Lap_h, periodic."""
    return (4.0 * x - neighbour_sum(x)) / (h * h)


def residual(f: np.ndarray, x: np.ndarray, h: float) -> np.ndarray:
    """r = f - A x (Algorithm 6)."""
    return f - apply_A(x, h)


def scaled_residual_exact(b: np.ndarray, x: np.ndarray) -> list:
    """Exact scaled residual b - (4 x - sum of the 4 periodic neighbours) of
    binary64 grids b and x (Algorithm 6's residual step in the scaled form
    h^2 f - h^2 A x), as Python Fractions: every binary64 value is a dyadic
    rational, so nothing is rounded.  Returned as a list of rows.  Slow; for
    small grids.  It fixes the value that any evaluation of the residual in
    finite precision approximates."""
    from fractions import Fraction
    n = x.shape[0]
    X = [[Fraction(float(v)) for v in row] for row in x]
    out = []
    for i in range(n):
        row = []
        for j in range(n):
            nb = X[(i - 1) % n][j] + X[(i + 1) % n][j] + X[i][(j - 1) % n] + X[i][(j + 1) % n]
            row.append(Fraction(float(b[i, j])) - (4 * X[i][j] - nb))
        out.append(row)
    return out


def red_mask(n: int) -> np.ndarray:
    """Boolean mask of red points, (i + j) even."""
    i = np.arange(n)
    return ((i[:, None] + i[None, :]) % 2) == 0


# ---------------------------------------------------------------------------
# Red-black Gauss-Seidel (Sec. 2.2; Algorithm 6 relaxation)
# ---------------------------------------------------------------------------

def rbgs_half_sweep(x: np.ndarray, f: np.ndarray, h: float, colour: int) -> None:
    """One colour of a Gauss-Seidel sweep, in place.

    Each point of the colour solves its own row of A x = f exactly:
    x_ij <- (h^2 f_ij + sum of 4 neighbours) / 4.  All neighbours of a point
    have the other colour, so updating the colour at once equals any
    sequential order within it.  colour 0 = red ((i + j) even), 1 = black.
    """
    mask = red_mask(x.shape[0])
    if colour == 1:
        mask = ~mask
    new = (h * h * f + neighbour_sum(x)) / 4.0
    x[mask] = new[mask]


def rbgs(x: np.ndarray, f: np.ndarray, h: float, sweeps: int) -> None:
    """`sweeps` red-black Gauss-Seidel sweeps (red half then black half)."""
    for _ in range(sweeps):
        rbgs_half_sweep(x, f, h, 0)
        rbgs_half_sweep(x, f, h, 1)


# ---------------------------------------------------------------------------
# Transfers
# ---------------------------------------------------------------------------

def restrict_fw(r: np.ndarray) -> np.ndarray:
    """Full-weighting restriction to the n/2 grid, periodic.

    r_c(I, J) = [4 r(2I, 2J) + 2 (edge neighbours) + (corner neighbours)] / 16
    with coarse node (I, J) at fine node (2I, 2J).
    """
    s = r
    edge = (np.roll(s, 1, 0) + np.roll(s, -1, 0) + np.roll(s, 1, 1) + np.roll(s, -1, 1))
    corner = (np.roll(np.roll(s, 1, 0), 1, 1) + np.roll(np.roll(s, 1, 0), -1, 1)
              + np.roll(np.roll(s, -1, 0), 1, 1) + np.roll(np.roll(s, -1, 0), -1, 1))
    full = (4.0 * s + 2.0 * edge + corner) / 16.0
    return np.ascontiguousarray(full[0::2, 0::2])


def _solve_cyclic_tridiagonal(a: float, b: float, c: float, d: np.ndarray) -> np.ndarray:
    """Solve the periodic tridiagonal systems a y_{k-1} + b y_k + c y_{k+1} = d_k.

    d has shape (m, L): L independent right-hand sides along axis 0.
    Sherman-Morrison on the Thomas algorithm: the two corner entries of the
    cyclic matrix are split off as a rank-one update u v^T.  Written for
    constant coefficients and m >= 3 unknowns.
    """
    m = d.shape[0]
    if m < 3:
        raise ValueError("cyclic tridiagonal solve needs at least 3 unknowns")
    gamma = -b
    diag = np.full(m, b, dtype=np.float64)
    diag[0] = b - gamma
    diag[-1] = b - a * c / gamma
    # forward-elimination factors (independent of the right-hand side)
    cp = np.empty(m)
    den = np.empty(m)
    den[0] = diag[0]
    cp[0] = c / diag[0]
    for k in range(1, m):
        den[k] = diag[k] - a * cp[k - 1]
        cp[k] = c / den[k]

    def thomas(rhs: np.ndarray) -> np.ndarray:
        dp = np.empty_like(rhs)
        dp[0] = rhs[0] / den[0]
        for k in range(1, m):
            dp[k] = (rhs[k] - a * dp[k - 1]) / den[k]
        y = np.empty_like(rhs)
        y[-1] = dp[-1]
        for k in range(m - 2, -1, -1):
            y[k] = dp[k] - cp[k] * y[k + 1]
        return y

    u = np.zeros(m)
    u[0] = gamma
    u[-1] = c  # the (last, first) corner entry of the cyclic matrix
    y = thomas(d)
    q = thomas(u[:, None])[:, 0]
    # v = (1, 0, ..., 0, a / gamma): v^T y picks up the (first, last) corner
    vy = y[0] + (a / gamma) * y[-1]
    vq = q[0] + (a / gamma) * q[-1]
    return y - q[:, None] * (vy / (1.0 + vq))[None, :]


def spline_midpoints(v: np.ndarray, H: float) -> np.ndarray:
    """Midpoints of the periodic cubic interpolating splines along axis 0.

    For each column of v (shape (m, L)), the spline's second derivatives M at
    the nodes solve the periodic system
    M_{k-1} + 4 M_k + M_{k+1} = (6 / H^2)(v_{k+1} - 2 v_k + v_{k-1});
    between nodes k and k+1 the spline's value at the midpoint is
    (v_k + v_{k+1}) / 2 - (H^2 / 16)(M_k + M_{k+1}).
    """
    rhs = (6.0 / (H * H)) * (np.roll(v, -1, 0) - 2.0 * v + np.roll(v, 1, 0))
    M = _solve_cyclic_tridiagonal(1.0, 4.0, 1.0, rhs)
    return 0.5 * (v + np.roll(v, -1, 0)) - (H * H / 16.0) * (M + np.roll(M, -1, 0))


def prolong_cubic_1d(v: np.ndarray, H: float) -> np.ndarray:
    """Refine periodic lines (axis 0) by 2: node I -> 2I, 2I+1 -> spline midpoint."""
    m = v.shape[0]
    out = np.empty((2 * m,) + v.shape[1:])
    out[0::2] = v
    vv = v if v.ndim == 2 else v[:, None]
    mid = spline_midpoints(vv, H)
    out[1::2] = mid if v.ndim == 2 else mid[:, 0]
    return out


def prolong_cubic(ec: np.ndarray) -> np.ndarray:
    """Tensor-product periodic cubic spline prolongation, (n/2)^2 -> n^2.

    Refines every coarse row along x, then every resulting column along y
    (the bivariate interpolating spline on a periodic tensor grid).
    """
    nc = ec.shape[0]
    H = grid_h(nc)
    rows = prolong_cubic_1d(ec.T, H).T        # along x: (nc, 2 nc)
    return np.ascontiguousarray(prolong_cubic_1d(rows, H))  # along y: (2 nc, 2 nc)


def spline_values(v: np.ndarray, H: float, factor: int) -> np.ndarray:
    """Periodic cubic interpolating splines along axis 0 (columns of v, node
    spacing H) evaluated at the points k + j / factor, j = 0 .. factor - 1, of
    every interval [k, k + 1]: with the nodes' second derivatives M (the
    periodic system of spline_midpoints) and t = j / factor,
    s = (1 - t) v_k + t v_{k+1} + (H^2 / 6) [((1 - t)^3 - (1 - t)) M_k + (t^3 - t) M_{k+1}]."""
    rhs = (6.0 / (H * H)) * (np.roll(v, -1, 0) - 2.0 * v + np.roll(v, 1, 0))
    M = _solve_cyclic_tridiagonal(1.0, 4.0, 1.0, rhs)
    vn, Mn = np.roll(v, -1, 0), np.roll(M, -1, 0)
    out = np.empty((factor * v.shape[0],) + v.shape[1:])
    for j in range(factor):
        t = j / factor
        out[j::factor] = ((1.0 - t) * v + t * vn
                          + (H * H / 6.0) * (((1.0 - t) ** 3 - (1.0 - t)) * M + (t ** 3 - t) * Mn))
    return out


def prolong_cubic_factor(ec: np.ndarray, factor: int) -> np.ndarray:
    """Tensor-product periodic cubic spline prolongation by `factor` (a power
    of two), (n / factor)^2 -> n^2: coarse node I -> fine factor * I, the spline
    evaluated at every fine point, rows (along x) then columns (along y).  The
    paper's two-level cycle interpolates the coarse correction by 16 in one
    step with a bivariate spline (Sec. 4.1; Table 1 N_step = 4)."""
    nc = ec.shape[0]
    H = grid_h(nc)
    rows = spline_values(ec.T, H, factor).T
    return np.ascontiguousarray(spline_values(rows, H, factor))


def restrict_fw_factor(r: np.ndarray, factor: int) -> np.ndarray:
    """Restriction by `factor` (a power of two) as repeated full weighting."""
    while factor > 1:
        r = restrict_fw(r)
        factor //= 2
    return r


def prolong_linear(ec: np.ndarray) -> np.ndarray:
    """Bilinear prolongation (textbook special case used to pin the V-cycle)."""
    nc = ec.shape[0]
    n = 2 * nc
    out = np.zeros((n, n))
    out[0::2, 0::2] = ec
    out[1::2, 0::2] = 0.5 * (ec + np.roll(ec, -1, 0))
    out[:, 1::2] = 0.5 * (out[:, 0::2] + np.roll(out[:, 0::2], -1, 1))
    return out


# ---------------------------------------------------------------------------
# Exact solutions (the plain definition x* = A^+ f)
# ---------------------------------------------------------------------------

def laplacian_eigenvalues(n: int, h: float) -> np.ndarray:
    """lambda(kx, ky) = (4 / h^2)(sin^2(pi kx / n) + sin^2(pi ky / n))."""
    k = np.arange(n)
    s = np.sin(np.pi * k / n) ** 2
    return (4.0 / (h * h)) * (s[:, None] + s[None, :])


def exact_solve_fft(f: np.ndarray, h: float | None = None) -> np.ndarray:
    """x* = A^+ f by diagonalising A with the 2D DFT (library FFT as a step).

    The periodic 5-point Laplacian's eigenvectors are the Fourier modes with
    eigenvalues lambda(k); the zero mode is dropped (zero-mean gauge).
    """
    n = f.shape[0]
    if h is None:
        h = grid_h(n)
    lam = laplacian_eigenvalues(n, h)
    fh = np.fft.fft2(f)
    lam[0, 0] = 1.0
    xh = fh / lam
    xh[0, 0] = 0.0
    return np.fft.ifft2(xh).real


def dense_operator(n: int, h: float) -> np.ndarray:
    """A as an explicit (n^2 x n^2) matrix, built point by point from the stencil."""
    N = n * n
    A = np.zeros((N, N))
    for i in range(n):
        for j in range(n):
            p = i * n + j
            A[p, p] += 4.0 / (h * h)
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                q = ((i + di) % n) * n + (j + dj) % n
                A[p, q] -= 1.0 / (h * h)
    return A


def gauss_solve(M: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Gaussian elimination with partial pivoting, written out."""
    M = M.astype(np.float64).copy()
    b = b.astype(np.float64).copy()
    m = M.shape[0]
    for k in range(m):
        p = k + int(np.argmax(np.abs(M[k:, k])))
        if p != k:
            M[[k, p]] = M[[p, k]]
            b[[k, p]] = b[[p, k]]
        piv = M[k, k]
        for i in range(k + 1, m):
            l = M[i, k] / piv
            if l != 0.0:
                M[i, k:] -= l * M[k, k:]
                b[i] -= l * b[k]
    x = np.zeros(m)
    for k in range(m - 1, -1, -1):
        x[k] = (b[k] - M[k, k + 1:] @ x[k + 1:]) / M[k, k]
    return x


def dense_solve(f: np.ndarray, h: float | None = None) -> np.ndarray:
    """x* by brute force: the bordered system [[A, 1], [1^T, 0]] [x; mu] = [f; 0].

    The border forces sum(x) = 0; mu absorbs the mean of f (zero for a
    compatible source).
    """
    n = f.shape[0]
    if h is None:
        h = grid_h(n)
    N = n * n
    A = dense_operator(n, h)
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = A
    B[:N, N] = 1.0
    B[N, :N] = 1.0
    rhs = np.zeros(N + 1)
    rhs[:N] = f.ravel()
    sol = gauss_solve(B, rhs)
    return sol[:N].reshape(n, n)


def coarse_solve(r: np.ndarray, h: float) -> np.ndarray:
    """Coarsest-grid exact solve e = A^+ (r - mean r) by the bordered dense system."""
    return dense_solve(r - r.mean(), h)


# ---------------------------------------------------------------------------
# V-cycle (Fig. 1a; Algorithm 6) and the solve loop
# ---------------------------------------------------------------------------

def vcycle(x: np.ndarray, f: np.ndarray, h: float, nu1: int = 2, nu2: int = 2,
           coarsest: int = 8, prolong=prolong_cubic) -> np.ndarray:
    """One V(nu1, nu2) cycle on A x = f, returning the new x.

    relax nu1 -> r = f - A x -> restrict -> recurse on A_2h e = r_2h from
    e = 0 (exact solve once the grid is coarsest x coarsest) -> x += P e ->
    relax nu2.
    """
    n = x.shape[0]
    x = x.copy()
    if n <= coarsest:
        return coarse_solve(f, h)
    rbgs(x, f, h, nu1)
    rc = restrict_fw(residual(f, x, h))
    ec = vcycle(np.zeros_like(rc), rc, 2.0 * h, nu1, nu2, coarsest, prolong)
    x += prolong(ec)
    rbgs(x, f, h, nu2)
    return x


def two_level_cycle(x: np.ndarray, f: np.ndarray, h: float, factor: int = 16, nu: int = 20,
                    coarse_sweeps: int = 10, prolong=None) -> np.ndarray:
    """One cycle of the paper's two-level scheme (Sec. 4.1; Algorithm 6 with a
    single coarse level): relax nu times (red-black Gauss-Seidel), restrict the
    residual by `factor`, relax the coarse correction equation coarse_sweeps
    times from zero (Algorithm 6's coarsest-level relaxation; 0 = the exact
    coarse solve), interpolate the correction back by `factor` with the cubic
    spline and add it.  No post-smoothing (Algorithm 6 relaxes before the
    coarse correction only).  `prolong`, when given, maps the coarse
    correction to the fine grid in place of the cubic spline by `factor` (the
    SR operator of Algorithm 5, for example)."""
    x = x.copy()
    rbgs(x, f, h, nu)
    rc = restrict_fw_factor(residual(f, x, h), factor)
    hc = h * factor
    if coarse_sweeps > 0:
        ec = np.zeros_like(rc)
        rbgs(ec, rc, hc, coarse_sweeps)
    else:
        ec = coarse_solve(rc, hc)
    return x + (prolong_cubic_factor(ec, factor) if prolong is None else prolong(ec))


def relative_residual(f: np.ndarray, x: np.ndarray, h: float) -> float:
    """||f - A x||_2 / ||f||_2 (discrete 2-norm)."""
    return float(np.linalg.norm(residual(f, x, h)) / np.linalg.norm(f))


def solve(f: np.ndarray, tol: float = 1e-10, max_cycles: int = 100,
          nu1: int = 2, nu2: int = 2, coarsest: int = 8, x0=None,
          prolong=prolong_cubic):
    """FP64 V-cycles until ||f - A x|| / ||f|| <= tol, then project to zero mean.

    Returns (x, info) with info = {cycles, rel_residual, update_norm, history}.
    A zero source returns x = 0 after zero cycles.
    """
    n = f.shape[0]
    h = grid_h(n)
    f = f - f.mean()
    x = np.zeros_like(f) if x0 is None else np.array(x0, dtype=np.float64)
    fnorm = np.linalg.norm(f)
    history = []
    cycles = 0
    upd = 0.0
    if fnorm == 0.0:
        return np.zeros_like(f), dict(cycles=0, rel_residual=0.0, update_norm=0.0,
                                       history=[])
    rel = relative_residual(f, x, h)
    history.append(rel)
    while rel > tol and cycles < max_cycles:
        xn = vcycle(x, f, h, nu1, nu2, coarsest, prolong)
        upd = float(np.linalg.norm(xn - x))
        x = xn
        cycles += 1
        rel = relative_residual(f, x, h)
        history.append(rel)
    x = x - x.mean()
    return x, dict(cycles=cycles, rel_residual=rel, update_norm=upd, history=history)
