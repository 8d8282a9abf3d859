"""Host logic of the generator's training data (no GPU).

The augmentation must be a symmetry of the whole V-cycle: the pair computed
from a transformed source equals the transformed pair.  The pair is computed
here with the oracle (smoothing, restriction, exact coarse and fine solves,
cubic prolongation), on a 32^2 grid, for every element of the square's
symmetry group combined with an even shift.
"""
import numpy as np
import pytest

from oracle import multigrid as omg

torch = pytest.importorskip("torch")


def _pair(f, nu=2):
    """Oracle pair (q, t) of one top-level coarse correction from x = 0."""
    n = f.shape[0]
    h = omg.grid_h(n)
    fz = f - f.mean()
    xs = omg.exact_solve_fft(fz, h)
    x = np.zeros_like(f)
    omg.rbgs(x, fz, h, nu)
    ef = xs - x
    ef -= ef.mean()
    rc = omg.restrict_fw(omg.residual(fz, x, h))
    ec = omg.exact_solve_fft(rc, 2 * h)
    s = np.abs(ec).max()
    return ec / s, (ef - omg.prolong_cubic(ec)) / s


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("flip", [False, True])
def test_augmentation_commutes_with_the_pair_construction(k, flip):
    from paper_2403_07936_gb300.train_sr import d4_index
    n = 32
    f = np.random.default_rng(k + 4 * flip).standard_normal((n, n))
    q, t = _pair(f)
    fy, fx = (a.numpy() for a in d4_index(n, k, flip))
    cy, cx = (a.numpy() for a in d4_index(n // 2, k, flip))
    sy, sx = 3, 5  # coarse shift, fine shift doubled
    f2 = np.roll(f[fy, fx], (2 * sy, 2 * sx), (0, 1))
    q2, t2 = _pair(f2)
    np.testing.assert_allclose(q2, np.roll(q[cy, cx], (sy, sx), (0, 1)), atol=1e-12)
    np.testing.assert_allclose(t2, np.roll(t[fy, fx], (2 * sy, 2 * sx), (0, 1)), atol=1e-11)


def test_augment_keeps_coarse_nodes_on_even_fine_nodes():
    from paper_2403_07936_gb300.train_sr import augment
    rng = np.random.default_rng(0)
    q = torch.tensor(rng.standard_normal((3, 8, 8)))
    t = torch.zeros((3, 16, 16), dtype=q.dtype)
    t[:, 0::2, 0::2] = q
    g = torch.Generator()
    g.manual_seed(1)
    for _ in range(16):
        q2, t2 = augment(q, t, g)
        assert torch.equal(t2[:, 0::2, 0::2], q2)
        assert torch.count_nonzero(t2[:, 1::2, :]) == 0 and torch.count_nonzero(t2[:, :, 1::2]) == 0
