"""Seeded synthetic pressure-Poisson sources (input generation only).

The paper solves the pressure-Poisson equation whose source is the divergence
of the advective term of a biperiodic turbulent velocity field with zero
viscosity (Sec. 3.2, Eq. poisson_ns, and Sec. 3.3 where nu = 0).  Its
Navier-Stokes data set is not public, so every input here is drawn from a
seeded spectrum that has the same structure:

* a divergence-free, biperiodic velocity u = (d_y psi, -d_x psi) on [0, 2 pi)^2,
* random-phase Fourier modes with energy spectrum E(k) ~ k^(-5/3) for
  1 <= |k| <= k_max, so |psi_hat(k)| ~ |k|^(-7/3),
* source f = -sum_ij (d_i u_j)(d_j u_i) = -(u_x^2 + 2 u_y v_x + v_y^2),
  the discrete mean removed (the periodic problem needs a zero-mean source).

The module holds no multigrid arithmetic: it is shared by the CPU oracle, the
tests and the benchmark purely as the input recipe.  Random numbers come from
the counter-based SplitMix64 generator (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), so every source is
reproducible from (n, k_max, seed) alone.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Return the first `count` outputs of SplitMix64 started at `seed`.

    Output i is mix(seed + (i + 1) * gamma) with the published finaliser.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (
            np.arange(1, count + 1, dtype=np.uint64) * _GAMMA)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """`count` doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def config_seed(config: int, item: int) -> int:
    """Seed of right-hand side `item` of workload `config` (1_000_003 c + i)."""
    return 1_000_003 * config + item


def default_kmax(n: int) -> int:
    """Forcing band edge k_max = n / 8 (k <= 8 at 64^2, k <= 256 at 2048^2)."""
    return max(1, n // 8)


def _streamfunction_hat(n: int, kmax: int, seed: int) -> np.ndarray:
    if not (1 <= kmax < n // 2):
        raise ValueError(f"k_max={kmax} must lie in [1, n/2) for n={n}")
    # Half-plane modes in a fixed order: ky outer (0..kmax), kx inner
    # (-kmax..kmax), keeping ky > 0 or (ky == 0 and kx > 0), 1 <= |k| <= kmax.
    ky, kx = np.meshgrid(np.arange(0, kmax + 1), np.arange(-kmax, kmax + 1), indexing="ij")
    ky, kx = ky.ravel(), kx.ravel()
    k2 = kx * kx + ky * ky
    keep = ((ky > 0) | (kx > 0)) & (k2 >= 1) & (k2 <= kmax * kmax)
    ky, kx, k2 = ky[keep], kx[keep], k2[keep]
    phases = 2.0 * np.pi * uniform01(seed, ky.size)
    c = k2.astype(np.float64) ** (-7.0 / 6.0) * np.exp(1j * phases)  # |k|^(-7/3) e^{i phi}
    psi_hat = np.zeros((n, n), dtype=np.complex128)
    psi_hat[ky % n, kx % n] = c
    psi_hat[(-ky) % n, (-kx) % n] = np.conj(c)
    return psi_hat


def turbulent_velocity(n: int, kmax: int, seed: int):
    """Seeded divergence-free velocity (u, v) with rms(|u|) = 1, shape (n, n).

    Arrays are indexed [iy, ix]; x runs along the contiguous axis.
    """
    psi_hat = _streamfunction_hat(n, kmax, seed)
    k = np.fft.fftfreq(n, d=1.0 / n)
    kx = k[None, :]
    ky = k[:, None]
    u_hat = 1j * ky * psi_hat
    v_hat = -1j * kx * psi_hat
    u = np.fft.ifft2(u_hat).real
    v = np.fft.ifft2(v_hat).real
    scale = 1.0 / np.sqrt(np.mean(u * u + v * v))
    return u * scale, v * scale, u_hat * scale, v_hat * scale


def turbulent_source(n: int, kmax: int | None = None, seed: int = 0) -> np.ndarray:
    """Pressure-Poisson source f = -(u_x^2 + 2 u_y v_x + v_y^2), zero mean, FP64.

    Derivatives are spectral; the product has wavenumbers up to 2 k_max <= n/4,
    so it is represented on the grid without aliasing.
    """
    if kmax is None:
        kmax = default_kmax(n)
    _, _, u_hat, v_hat = turbulent_velocity(n, kmax, seed)
    k = np.fft.fftfreq(n, d=1.0 / n)
    kx = k[None, :]
    ky = k[:, None]
    ux = np.fft.ifft2(1j * kx * u_hat).real
    uy = np.fft.ifft2(1j * ky * u_hat).real
    vx = np.fft.ifft2(1j * kx * v_hat).real
    vy = np.fft.ifft2(1j * ky * v_hat).real
    f = -(ux * ux + 2.0 * uy * vx + vy * vy)
    f -= f.mean()
    return np.ascontiguousarray(f)


def perturb_with(f_prev: np.ndarray, g: np.ndarray, eps: float = 0.01) -> np.ndarray:
    """f + eps (|f| / |g|) g with the mean removed."""
    f = f_prev + eps * (np.linalg.norm(f_prev) / np.linalg.norm(g)) * g
    f -= f.mean()
    return np.ascontiguousarray(f)


def perturbed_source(f_prev: np.ndarray, seed: int, eps: float = 0.01) -> np.ndarray:
    """Next source of a serving stream: f + eps (|f| / |g|) g, g a fresh source."""
    n = f_prev.shape[0]
    return perturb_with(f_prev, turbulent_source(n, default_kmax(n), seed), eps)
