"""Pins of the windowed SR oracle (Sec. 3.1, Fig. 2; Algorithms 1-5): the
symmetric-log normalisation by its fixed points and closed forms, and the
window stitching by exactness for operators whose receptive field stays
inside the ghost margin and by shift equivariance (CPU)."""
import numpy as np
import pytest

from oracle import generator as og
from oracle import windowed as ow
from synthetic.weights import random_weights

P_MIN, P_MAX = 1e-10, 1e-3  # the paper's normalisation interval


def _nearest(f):
    return lambda w: np.kron(w, np.ones((f, f)))


def _blur(x, padding, times):
    k = np.ones((1, 1, 3, 3)) / 9.0
    y = x[None]
    for _ in range(times):
        y = og.conv3x3(y, k, np.zeros(1), padding)
    return y[0]


def test_linear_maps_are_inverse_for_the_unit_target():
    rng = np.random.default_rng(0)
    p = rng.uniform(-12, -1, 50)
    u, v = -10.0, -3.0
    q = ow.linear_normalize(p, u, v, 0.0, 1.0)
    np.testing.assert_allclose(ow.linear_denormalize(q, u, v, 0.0, 1.0), p, rtol=0, atol=1e-13)
    assert ow.linear_normalize(u, u, v, 0.0, 1.0) == 0.0 and ow.linear_normalize(v, u, v, 0.0, 1.0) == 1.0


def test_symlog_fixes_the_ends_the_sign_and_the_log_midpoint():
    T = lambda p: ow.symlog_normalize(p, P_MIN, P_MAX)  # noqa: E731
    assert T(P_MIN) == 0.0 and T(P_MAX) == 1.0 and T(-P_MAX) == -1.0 and T(0.0) == 0.0
    np.testing.assert_allclose(T(np.sqrt(P_MIN * P_MAX)), 0.5, atol=1e-15)
    np.testing.assert_allclose(T(-np.sqrt(P_MIN * P_MAX)), -0.5, atol=1e-15)
    assert T(10 * P_MAX) == 1.0 and T(P_MIN / 10) == 0.0  # clamped magnitudes
    x = np.geomspace(P_MIN, P_MAX, 200)
    assert np.all(np.diff(T(x)) > 0)


def test_symlog_round_trip():
    rng = np.random.default_rng(1)
    p = np.power(10.0, rng.uniform(-10, -3, (16, 16))) * rng.choice([-1.0, 1.0], (16, 16))
    q = ow.symlog_normalize(p, P_MIN, P_MAX)
    assert np.all(np.abs(q) <= 1.0)
    np.testing.assert_allclose(ow.symlog_denormalize(q, P_MIN, P_MAX), p, rtol=1e-12, atol=0)
    assert ow.symlog_denormalize(0.0, P_MIN, P_MAX) == 0.0


@pytest.mark.parametrize("factor", [2, 4])
def test_stitching_a_pointwise_upsampler_is_exact(factor):
    q = np.random.default_rng(2).standard_normal((16, 16))
    got = ow.windowed_upsample(q, _nearest(factor), factor)
    np.testing.assert_array_equal(got, np.kron(q, np.ones((factor, factor))))


@pytest.mark.parametrize("times,exact", [(1, True), (2, True), (3, False)])
def test_windows_are_exact_within_the_ghost_margin(times, exact):
    """A 3x3 blur applied `times` times reaches `times` cells; the kept block is
    2 cells inside a 6-cell window, so up to two blurs see exactly what the
    whole periodic grid would show them, and a third reaches the zero padding."""
    q = np.random.default_rng(3).standard_normal((16, 16))
    up = lambda w: np.kron(_blur(w, "zero", times), np.ones((2, 2)))  # noqa: E731
    got = ow.windowed_upsample(q, up, 2)
    ref = np.kron(_blur(q, "circular", times), np.ones((2, 2)))
    if exact:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    else:
        assert np.abs(got - ref).max() > 1e-3


def test_windowed_generator_commutes_with_shifts_by_the_window_stride():
    """Shifting the coarse field by whole window steps (2 cells) only relabels
    the windows, so the output shifts by the same steps times the factor."""
    w = random_weights(4, n_blocks=1)
    gen = lambda win: og.generator_forward(win, w, n_blocks=1, padding="zero")  # noqa: E731
    ec = np.random.default_rng(5).standard_normal((12, 12)) * 1e-5
    out = ow.windowed_sr_prolong(ec, gen, 2, P_MIN, P_MAX)
    assert out.shape == (24, 24) and np.all(np.isfinite(out))
    shifted = ow.windowed_sr_prolong(np.roll(ec, (2, 4), axis=(0, 1)), gen, 2, P_MIN, P_MAX)
    np.testing.assert_allclose(shifted, np.roll(out, (4, 8), axis=(0, 1)), rtol=1e-12, atol=0)


def test_windowed_prolongation_maps_back_to_the_input_scale():
    rng = np.random.default_rng(6)
    ec = np.power(10.0, rng.uniform(-9, -4, (8, 8))) * rng.choice([-1.0, 1.0], (8, 8))
    got = ow.windowed_sr_prolong(ec, _nearest(2), 2, P_MIN, P_MAX)
    np.testing.assert_allclose(got, np.kron(ec, np.ones((2, 2))), rtol=1e-12, atol=0)
