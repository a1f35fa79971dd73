"""The seeded synthetic inputs follow their stated recipe (no GPU).

Both the CUDA path and the oracle are fed from paper_1907_11771_gb300.inputs, so
its recipe is part of every parity claim: the same seed gives the same arrays,
the media stay in 1 + [0, 0.5 * n_gauss] and are periodic and smooth, the pulse
sits where it is placed, the batch draws its sides from the stated set, and the
receivers lie on the row y = 3N/4.
"""
import numpy as np
import pytest

from paper_1907_11771_gb300 import inputs


def test_same_seed_same_arrays_other_seed_other_arrays():
    a = inputs.acoustic_problem((48, 40), 5, 16, 6.0)
    b = inputs.acoustic_problem((48, 40), 5, 16, 6.0)
    c = inputs.acoustic_problem((48, 40), 6, 16, 6.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[1], c[1])
    # kappa and rho come from different seeds
    assert not np.array_equal(a[1], a[2])


@pytest.mark.parametrize("shape,n_gauss", [((64, 96), 16), ((20, 24, 28), 64)])
def test_media_bounds_positivity_and_periodicity(shape, n_gauss):
    m = inputs.smooth_media(shape, n_gauss, 3)
    assert m.shape == shape
    assert m.min() >= 1.0 and m.max() <= 1.0 + 0.5 * n_gauss
    assert m.max() > 1.0
    # periodic Gaussians: the wrap-around difference is as small as an interior one
    # (widths >= N/32 cells keep neighbouring values close everywhere)
    for ax in range(len(shape)):
        inner = np.abs(np.diff(m, axis=ax)).max()
        wrap = np.abs(np.take(m, 0, axis=ax) - np.take(m, -1, axis=ax)).max()
        assert wrap <= 1.5 * inner + 1e-15


def test_const_rho_and_fields():
    y0, kappa, rho = inputs.acoustic_problem((32, 36), 1, 16, 4.0, const_rho=True)
    assert y0.shape == (3, 32, 36)
    assert np.all(rho == 1.0)
    assert np.all(y0[1:] == 0.0)
    y3, _, _ = inputs.acoustic_problem((16, 18, 20), 1, 64, 4.0, n_pulses=3, centred=False)
    assert y3.shape == (4, 16, 18, 20)
    assert np.all(y3[1:] == 0.0)


def test_centred_pulse_peak_and_symmetry():
    n = 64
    y0, _, _ = inputs.acoustic_problem((n, n), 0, 16, 5.0)
    p = y0[0]
    assert np.unravel_index(np.argmax(p), p.shape) == (n // 2, n // 2)
    assert p[n // 2, n // 2] == pytest.approx(1.0, abs=1e-12)
    # exp(-r^2 / (2 sigma^2)) at one sigma along x
    assert p[n // 2, n // 2 + 5] == pytest.approx(np.exp(-0.5), rel=1e-12)
    # symmetric about the centre on the periodic grid
    assert np.allclose(p[n // 2, n // 2 + 1:], p[n // 2, n // 2 - 1:0:-1][:n // 2 - 1], rtol=0, atol=1e-15)


def test_wave1d_initial_condition():
    y, dx = inputs.wave1d_initial(256)
    x = 2 * np.pi * np.arange(256) / 256
    assert dx == pytest.approx(2 * np.pi / 256)
    assert np.allclose(y[0], np.exp(-20 * (x - np.pi) ** 2), rtol=0, atol=0)
    assert np.all(y[1] == 0.0)


def test_batch_sides_come_from_the_stated_set():
    sides = inputs.batch_sides()
    assert len(sides) == 256
    choices = (128, 256, 384, 512, 768, 1024)
    assert set(sides) <= set(choices)
    counts = np.array([sides.count(c) for c in choices])
    # uniform draw: every side occurs, none far from 256/6
    assert counts.min() > 20 and counts.max() < 70
    assert sides == inputs.batch_sides()


def test_line_receivers():
    n = 1024
    r = inputs.line_receivers(n)
    assert r.dtype == np.int64 and len(r) == 64
    assert len(set(r.tolist())) == 64
    rows, cols = r // n, r % n
    assert np.all(rows == 3 * n // 4)
    assert cols[0] == 8 and np.all(np.diff(cols) == 16)
