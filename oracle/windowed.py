"""Plain FP64 CPU oracle of the windowed SR prolongation with symmetric-log
normalisation (Sec. 3.1 and Fig. 2; Appendix A, Algorithms 1-5).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product library.

The paper feeds its generator small windows of the coarse field instead of
the whole grid: the coarse values are normalised by a symmetric logarithm,
cut into overlapping n_s x n_s windows whose origins step by 2, each window
is super-resolved on its own, only the up-sampled central 2 x 2 block of
every window is kept, and the stitched field is mapped back.  The kept block
lies (n_s - 2) / 2 coarse cells inside its window, so an operator whose
receptive field reaches no further than that sees the same values it would
see on the whole grid (the paper's "ghost cells").

Readings where the paper is silent or inconsistent:
- Algorithm 1 as printed scales without adding the target offset a; only
  a = 0, b = 1 is used, where it and Algorithm 2 are exact inverses.
- Algorithm 3 maps log10|p| from [log10 p_min, log10 p_max] to [0, 1] and
  multiplies by sgn p.  Magnitudes outside [p_min, p_max] are clamped to the
  interval first (a magnitude below p_min would otherwise map below 0 and
  flip the sign); p = 0 stays 0.
- Algorithm 4 multiplies by the sign of the coarse input, which has other
  points than the fine output; here each fine value takes the sign of its
  own normalised value: p = sgn(q) 10^(log10 p_min + |q| (log10 p_max -
  log10 p_min)), and q = 0 gives 0.
- The fields are periodic, so windows wrap around the grid and every coarse
  point lies in exactly one kept block (no edge filling is needed).
- The up-sampler maps an n_s x n_s window to (r n_s) x (r n_s) for the
  refinement factor r (the paper's generator enlarges by 4 and is applied
  twice; the library's enlarges by 2); its output replaces the
  prolongation (Algorithm 5 has no spline term).
"""
from __future__ import annotations

import numpy as np


def linear_normalize(p, u: float, v: float, a: float, b: float):
    """Algorithm 1: (p - u) (b - a) / (v - u)."""
    return (np.asarray(p, dtype=np.float64) - u) * ((b - a) / (v - u))


def linear_denormalize(q, u: float, v: float, a: float, b: float):
    """Algorithm 2: (q - a) (v - u) / (b - a) + u."""
    return (np.asarray(q, dtype=np.float64) - a) * ((v - u) / (b - a)) + u


def symlog_normalize(p, p_min: float, p_max: float) -> np.ndarray:
    """Algorithm 3: sgn(p) T'(|p|), T' the linear map of log10 |p| from
    [log10 p_min, log10 p_max] to [0, 1] (magnitudes clamped to the interval)."""
    p = np.asarray(p, dtype=np.float64)
    mag = np.clip(np.abs(p), p_min, p_max)
    t = linear_normalize(np.log10(mag), np.log10(p_min), np.log10(p_max), 0.0, 1.0)
    return np.sign(p) * t


def symlog_denormalize(q, p_min: float, p_max: float) -> np.ndarray:
    """Algorithm 4 (sign taken from q itself): sgn(q) 10^(linear
    denormalisation of |q|)."""
    q = np.asarray(q, dtype=np.float64)
    lg = linear_denormalize(np.abs(q), np.log10(p_min), np.log10(p_max), 0.0, 1.0)
    return np.sign(q) * np.power(10.0, lg)


def windowed_upsample(q: np.ndarray, upsampler, factor: int, n_s: int = 6, core: int = 2) -> np.ndarray:
    """Algorithm 5's window loop on a periodic field q (n x n): window (a, b)
    covers coarse rows 2a - m .. 2a - m + n_s - 1 (m = (n_s - core) / 2, indices
    mod n) and likewise columns; upsampler(window) is (factor n_s)^2 and its
    central (factor core)^2 block becomes fine rows factor 2a .. factor (2a + core) - 1."""
    n = q.shape[0]
    if q.shape != (n, n) or n % core or (n_s - core) % 2 or core != 2:
        raise ValueError("square field, n a multiple of the core, core 2, n_s - core even")
    m = (n_s - core) // 2
    out = np.empty((factor * n, factor * n))
    idx = np.arange(n_s)
    for a in range(n // core):
        rows = (core * a - m + idx) % n
        for b in range(n // core):
            cols = (core * b - m + idx) % n
            w = q[np.ix_(rows, cols)]
            up = np.asarray(upsampler(w), dtype=np.float64)
            if up.shape != (factor * n_s, factor * n_s):
                raise ValueError(f"upsampler returned {up.shape}, expected {(factor * n_s,) * 2}")
            keep = up[factor * m:factor * (m + core), factor * m:factor * (m + core)]
            out[factor * core * a:factor * core * (a + 1), factor * core * b:factor * core * (b + 1)] = keep
    return out


def windowed_sr_prolong(ec: np.ndarray, upsampler, factor: int, p_min: float, p_max: float,
                        n_s: int = 6, core: int = 2) -> np.ndarray:
    """Algorithm 5: normalise, super-resolve every window, stitch the kept
    blocks, map back."""
    q = symlog_normalize(ec, p_min, p_max)
    return symlog_denormalize(windowed_upsample(q, upsampler, factor, n_s, core), p_min, p_max)
