"""The one-way wave with spectral derivatives (Sec. 4), oracle side.

Pins:
* the spectral derivative is exact on every resolved Fourier mode (closed forms of d/dx of
  sin and cos), and the Nyquist mode gets zero;
* Sec. 4's run (u0 = (1 - cos 2 pi x) / 2, lambda = dt/dx = 0.99 ISB / pi, once around the
  interval): the oracle's GBS run equals an independent 50-digit evaluation of R(xi)^M on the
  single excited mode (xi = -2 pi i dt) to FP64 rounding, and the error converges with order
  p (8 for GBS_8,6, 12 for GBS_12,8) until it meets the FP64 rounding floor of the whole run,
  FFTs included, about 1e-16 sum|c_k| per macro-step: 1e-13 for GBS_8,6 and 1e-12 for GBS_12,8
  at the finest levels (the paper reports coefficient-truncation floors of 1e-14 and 1e-12);
* those coefficient-truncation floors themselves, at 60 digits with everything exact but the
  weights: the error levels off at M |sum_k c~_k - 1| / 2, and with the weights chopped to FP64
  it sits at the paper's 1e-14 (GBS_8,6) and 1e-12 (GBS_12,8).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import gbs as OG
from oracle import mol as OM
from oracle import weights as OW
from paper_1907_11771_gb300 import schemes as S

ISB = {"GBS_8,6": 17.65320, "GBS_12,8": 22.06133}


def _weights(s):
    return OW.scheme_weights(s.order, list(s.steps_dep), list(s.steps_free), [Fraction(t) for t in s.c_free_text])


def test_spectral_derivative_is_exact_on_resolved_modes():
    n, L = 64, 1.0
    dx = L / n
    x = np.arange(n) * dx
    for m in (1, 2, 7, 31):
        k = 2 * np.pi * m / L
        for u, du in ((np.sin(k * x), k * np.cos(k * x)), (np.cos(k * x), -k * np.sin(k * x))):
            f = OM.rhs_oneway_spectral(u[None, :], dx)[0]
            assert np.max(np.abs(f + du)) <= 1e-12 * k
    nyq = (-1.0) ** np.arange(n)
    assert np.max(np.abs(OM.rhs_oneway_spectral(nyq[None, :], dx))) <= 1e-12
    const = np.full((1, n), 3.0)
    assert np.max(np.abs(OM.rhs_oneway_spectral(const, dx))) <= 1e-12


def _paper_run(scheme, n):
    steps, c = _weights(scheme)
    dx = 1.0 / n
    M = int(np.ceil(1.0 / (0.99 / np.pi * ISB[scheme.name] * dx)))
    dt = 1.0 / M
    x = np.arange(n) * dx
    u0 = 0.5 * (1 - np.cos(2 * np.pi * x))
    u = OG.gbs_run(lambda v: OM.rhs_oneway_spectral(v, dx), u0[None, :], dt, steps, OW.to_fp64(c), M)[0]
    return steps, c, M, np.max(np.abs(u - u0))


@pytest.mark.parametrize("scheme", [S.GBS_8_6, S.GBS_12_8])
def test_section4_run_matches_a_high_precision_single_mode_evaluation(scheme):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rows = []
    for n in (16, 32, 64, 256, 1024):
        steps, c, M, err = _paper_run(scheme, n)
        xi = mpmath.mpc(0, -2) * mpmath.pi / M
        R = mpmath.mpc(0)
        for N, ck in zip(steps, c):
            z = xi / N
            ym, yc = mpmath.mpc(1), 1 + z
            prev = ym
            for _ in range(N):
                prev, ym, yc = ym, yc, ym + 2 * z * yc
            R += mpmath.mpf(ck.numerator) / ck.denominator * (prev + 2 * ym + yc) / 4
        # u = 1/2 - (e^{2 pi i x} + e^{-2 pi i x}) / 4: mode 1 (amplitude 1/4) and its conjugate
        # are multiplied by R^M and its conjugate, so u_M - u_0 = -Re((R^M - 1) e^{2 pi i x}) / 2;
        # the error is its largest modulus over the grid points
        z = R ** M - 1
        pred = max(float(abs(mpmath.re(z * mpmath.expjpi(2 * mpmath.mpf(j) / n)))) / 2 for j in range(n))
        rows.append((n, err, pred))
        # FP64 rounding of the whole run, FFTs included: each macro-step adds about u sum|c_k|
        floor = 1e-16 * float(sum(abs(v) for v in c)) * M
        assert abs(err - pred) <= max(1e-2 * pred, floor), (n, err, pred)
    # order of convergence on the coarse levels, where the time error dominates (order 8: M = 3
    # and 6 at n = 16 and 32; order 12 reaches the rounding floor already at n = 32)
    if scheme.order == 8:
        rate = np.log2(rows[0][1] / rows[1][1])
        assert abs(rate - 8) < 0.6, rate
    # the finest level sits on the rounding floor, far above its own time error
    assert rows[-1][2] < 1e-18 and rows[-1][1] < 1e-11


@pytest.mark.parametrize("scheme,n,paper_floor", [(S.GBS_8_6, 1024, 1e-14), (S.GBS_12_8, 2048, 1e-12)])
def test_section4_coefficient_truncation_floors(scheme, n, paper_floor):
    """Sec. 4: with the weights truncated to FP64 the error stops converging, at 1e-14 (order 8)
    and 1e-12 (order 12); twenty significant digits of the weights reach 1e-16.  On the single
    excited mode of Sec. 4's run the error after one trip is |R(xi)^M - e^(-2 pi i)| / 2,
    evaluated here at 60 digits with everything exact but the weights.  With exact weights it
    keeps converging.  With FP64 weights it levels off at M |sum_k c~_k - 1| / 2, which grows
    with M: the weights' sum misses 1 by their rounding, and P_k(0) = 1.  Chopped toward zero,
    as "truncation" says, the weights put it at the paper's levels at these resolutions (within
    a factor of 3); rounded to nearest, as this library does, it is lower for GBS_12,8."""
    import math
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    steps, c = _weights(scheme)
    chop = []
    for v in c:
        f = float(v)
        if abs(Fraction(f)) > abs(v):
            f = math.nextafter(f, 0.0)
        chop.append(Fraction(f))
    near = [Fraction(float(v)) for v in c]
    lam = 0.99 * ISB[scheme.name] / math.pi
    M = math.ceil(n / lam)
    xi = mpmath.mpc(0, -2) * mpmath.pi / M
    target = mpmath.exp(mpmath.mpc(0, -2) * mpmath.pi)

    def err(cw):
        acc = mpmath.mpc(0)
        for a in reversed(OW.stability_poly(steps, cw)):
            acc = acc * xi + mpmath.mpf(a.numerator) / a.denominator
        return float(abs(acc ** M - target) / 2)

    assert err(c) <= 1e-4 * paper_floor                     # exact weights: still converging
    for cw in (chop, near):
        drift = M * abs(float(sum(cw) - 1)) / 2
        assert abs(err(cw) - drift) <= 0.05 * drift         # the floor is the weights' sum
    assert paper_floor / 3 <= err(chop) <= 3 * paper_floor
