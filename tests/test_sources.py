"""Checks of the seeded synthetic source recipe (no GPU)."""
import numpy as np

from synthetic.sources import (config_seed, perturbed_source, splitmix64, turbulent_source,
                               turbulent_velocity)


def test_splitmix64_published_vector():
    # First outputs of SplitMix64 seeded with 0 (reference sequence of the
    # published algorithm, as used to seed xoshiro generators).
    out = splitmix64(0, 3)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_source_reproducible_and_zero_mean():
    a = turbulent_source(64, 8, config_seed(0, 0))
    b = turbulent_source(64, 8, config_seed(0, 0))
    c = turbulent_source(64, 8, config_seed(0, 1))
    np.testing.assert_array_equal(a, b)
    assert np.abs(a - c).max() > 1e-3
    assert abs(a.mean()) < 1e-12 * np.abs(a).max()


def test_velocity_divergence_free_and_spectrum():
    n, kmax = 64, 8
    u, v, uh, vh = turbulent_velocity(n, kmax, 5)
    k = np.fft.fftfreq(n, d=1.0 / n)
    div = k[None, :] * uh + k[:, None] * vh
    assert np.abs(div).max() < 1e-9 * np.abs(uh).max()
    assert abs(np.mean(u * u + v * v) - 1.0) < 1e-12
    # per-mode energy |u_hat|^2 + |v_hat|^2 ~ |k|^(2 - 14/3) = |k|^(-8/3)
    e = np.abs(uh) ** 2 + np.abs(vh) ** 2
    k2 = k[None, :] ** 2 + k[:, None] ** 2
    sel = (k2 >= 1) & (k2 <= kmax * kmax)
    ratio = e[sel] / k2[sel] ** (-4.0 / 3.0)
    assert ratio.std() < 1e-9 * ratio.mean()
    assert not e[~sel].any()


def test_source_is_minus_divergence_of_advection():
    """f = -div((u.grad) u) for divergence-free u (an identity, checked spectrally)."""
    n, kmax = 64, 8
    u, v, uh, vh = turbulent_velocity(n, kmax, 11)
    k = np.fft.fftfreq(n, d=1.0 / n)
    dx = lambda a: np.fft.ifft2(1j * k[None, :] * np.fft.fft2(a)).real
    dy = lambda a: np.fft.ifft2(1j * k[:, None] * np.fft.fft2(a)).real
    adv_u = u * dx(u) + v * dy(u)
    adv_v = u * dx(v) + v * dy(v)
    f_ref = -(dx(adv_u) + dy(adv_v))
    f_ref -= f_ref.mean()
    np.testing.assert_allclose(turbulent_source(n, kmax, 11), f_ref,
                               atol=1e-9 * np.abs(f_ref).max())


def test_perturbed_source_is_one_percent():
    f = turbulent_source(32, 4, 1)
    g = perturbed_source(f, 2, 0.01)
    assert abs(np.linalg.norm(g - f) / np.linalg.norm(f) - 0.01) < 1e-3
