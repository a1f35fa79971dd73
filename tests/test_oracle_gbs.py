"""Pins for the oracle's GBS macro-step, its adjoint and the receiver misfit (no GPU).

* Dahlquist's test equation: one macro-step multiplies y by R(H lambda) where R is
  the stability polynomial (Appendix A, Appendix B) evaluated directly.
* Constant-coefficient periodic problems: every Fourier mode is multiplied by
  R(H lambda_k) with lambda_k from the closed-form stencil symbol.
* Order of accuracy: halving H divides the time error by about 2^p (Sec. 2.1, 3.2).
* The 1D wave problem against d'Alembert's solution and its spatial refinement.
* The stability edge at 0.99 / 1.01 x ISB / rho(A) (Sec. 2.2, Appendix A.1).
* Adjoint: dot-product identity and central finite differences of the gradient.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import gbs as G
from oracle import mol
from oracle import weights as W
from paper_1907_11771_gb300 import inputs
from tests.conftest import load_golden
from tests.test_oracle_mol import SYMBOL

SCHEMES = load_golden("paper_schemes.txt")


def scheme(name):
    sc = SCHEMES[name]
    dep = [int(t) for t in sc["dep"].split()]
    free = [int(t) for t in sc.get("free", "").split()]
    cf = [Fraction(t) for t in sc.get("cfree", "").split()]
    steps, c = W.scheme_weights(int(sc["order"]), dep, free, cf)
    return int(sc["order"]), steps, c


SQ8 = (8, [2, 4, 6, 8], W.square_weights([2, 4, 6, 8], 8))


@pytest.mark.parametrize("name", ["table1_order8", "gbs_8_6", "gbs_12_8", "gbs_8_8"])
def test_dahlquist_macro_step_equals_stability_polynomial(name):
    order, steps, c = scheme(name)
    R = [float(a) for a in W.stability_poly(steps, c)]
    cf = W.to_fp64(c)
    for lam in (1j * 0.7, -0.3 + 2.1j, 0.05 - 1.3j):
        for H in (0.5, 3.0):
            y0 = np.array([1.0 + 0.5j])
            out = G.gbs_macro_step(lambda y: lam * y, y0, H, steps, cf)
            expect = W.poly_eval(R, H * lam) * y0[0]
            assert out[0] == pytest.approx(expect, rel=1e-11)


def test_wave1d_modes_follow_R():
    # u + v is transported by +D and u - v by -D; each Fourier mode of w = u + v is
    # multiplied by R(i H s_k / dx) per macro-step, z = u - v by R(-i H s_k / dx).
    n, order = 64, 4
    dx = 2 * np.pi / n
    _, steps, c = scheme("gbs_8_6")
    R = [float(a) for a in W.stability_poly(steps, c)]
    rng = np.random.default_rng(0)
    y0 = rng.standard_normal((2, n))
    H = 0.05
    out = G.gbs_macro_step(lambda y: mol.rhs_wave1d(y, dx, order), y0, H, steps, W.to_fp64(c))
    th = 2 * np.pi * np.fft.fftfreq(n)
    s = SYMBOL[order](th) / dx
    Rp = np.array([W.poly_eval(R, 1j * H * sk) for sk in s])
    Rm = np.array([W.poly_eval(R, -1j * H * sk) for sk in s])
    w_in, z_in = np.fft.fft(y0[0] + y0[1]), np.fft.fft(y0[0] - y0[1])
    w_out, z_out = np.fft.fft(out[0] + out[1]), np.fft.fft(out[0] - out[1])
    np.testing.assert_allclose(w_out, Rp * w_in, atol=1e-11 * np.abs(w_in).max())
    np.testing.assert_allclose(z_out, Rm * z_in, atol=1e-11 * np.abs(z_in).max())


@pytest.mark.parametrize("order", [4, 6])
def test_acoustic2d_constant_coefficient_modes_follow_matrix_R(order):
    # y_out_k = R(H A_k) y_in_k with the 3x3 symbol matrix A_k of the acoustic operator.
    n, kappa0, b0 = 16, 1.5, 0.8
    dx = [1.0, 1.0]
    _, steps, c = SQ8
    R = [float(a) for a in W.stability_poly(steps, c)]
    kappa = np.full((n, n), kappa0)
    b = np.full((n, n), b0)
    rng = np.random.default_rng(4)
    y0 = rng.standard_normal((3, n, n))
    H = 0.3
    out = G.gbs_macro_step(lambda y: mol.rhs_acoustic(y, kappa, b, dx, order), y0, H, steps, W.to_fp64(c))
    Yin = np.fft.fft2(y0, axes=(1, 2))
    Yout = np.fft.fft2(out, axes=(1, 2))
    th = 2 * np.pi * np.fft.fftfreq(n)
    for ky in range(n):
        for kx in range(n):
            sx, sy = SYMBOL[order](th[kx]) / dx[0], SYMBOL[order](th[ky]) / dx[1]
            A = np.array([[0, -kappa0 * 1j * sx, -kappa0 * 1j * sy],
                          [-b0 * 1j * sx, 0, 0],
                          [-b0 * 1j * sy, 0, 0]])
            M = np.zeros((3, 3), complex)
            P = np.eye(3, dtype=complex)
            for a in R:
                M += a * P
                P = P @ (H * A)
            np.testing.assert_allclose(Yout[:, ky, kx], M @ Yin[:, ky, kx], atol=1e-10 * np.abs(Yin).max())


def _semi_discrete_exact(y0, t, n, order):
    dx = 2 * np.pi / n
    th = 2 * np.pi * np.fft.fftfreq(n)
    s = SYMBOL[order](th) / dx
    W_ = np.fft.fft(y0[0] + y0[1]) * np.exp(1j * s * t)
    Z_ = np.fft.fft(y0[0] - y0[1]) * np.exp(-1j * s * t)
    w, z = np.fft.ifft(W_).real, np.fft.ifft(Z_).real
    return np.stack([(w + z) / 2, (w - z) / 2])


def test_order_of_accuracy_by_refining_H():
    n, order = 256, 4
    y0, dx = inputs.wave1d_initial(n)
    _, steps, c = SQ8
    cf = W.to_fp64(c)
    T = 0.5
    errs = []
    for M in (8, 16):
        y = G.gbs_run(lambda y: mol.rhs_wave1d(y, dx, order), y0, T / M, steps, cf, M)
        ex = _semi_discrete_exact(y0, T, n, order)
        errs.append(np.linalg.norm(y - ex) / np.linalg.norm(ex))
    ratio = errs[0] / errs[1]
    assert 2 ** 7.5 < ratio < 2 ** 8.5, ratio


@pytest.mark.slow
def test_wave1d_against_dalembert_and_spatial_refinement():
    # At t = 2 pi the exact PDE solution is the initial state again (d'Alembert, periodic).
    # With H = 0.8 x the stability limit the error is dominated by the 4th-order FD error,
    # which drops by ~2^4 when the grid is refined.
    _, steps, c = SQ8
    cf = W.to_fp64(c)
    isb = W.isb_exact(W.stability_poly(steps, c))
    errs = []
    for n in (128, 256):
        y0, dx = inputs.wave1d_initial(n)
        rho = mol.symbol_max(4) / dx
        M = int(np.ceil(2 * np.pi / (0.8 * isb / rho)))
        y = G.gbs_run(lambda y: mol.rhs_wave1d(y, dx, 4), y0, 2 * np.pi / M, steps, cf, M)
        err_total = np.linalg.norm(y - y0) / np.linalg.norm(y0)
        semi = _semi_discrete_exact(y0, 2 * np.pi, n, 4)
        err_time = np.linalg.norm(y - semi) / np.linalg.norm(semi)
        assert err_time < 0.01 * err_total
        errs.append(err_total)
    assert 2 ** 3.5 < errs[0] / errs[1] < 2 ** 4.5


@pytest.mark.parametrize("factor,grows", [(0.99, False), (1.01, True)])
def test_stability_edge(factor, grows):
    n, order = 64, 4
    dx = 2 * np.pi / n
    _, steps, c = scheme("gbs_8_6")
    cf = W.to_fp64(c)
    isb = W.isb_exact(W.stability_poly(steps, c))
    th = 2 * np.pi * np.fft.fftfreq(n)
    rho = np.max(np.abs(SYMBOL[order](th))) / dx          # exact spectral radius on this grid
    H = factor * isb / rho
    rng = np.random.default_rng(7)
    y = rng.standard_normal((2, n))
    n0 = np.linalg.norm(y)
    for _ in range(120):
        y = G.gbs_macro_step(lambda v: mol.rhs_wave1d(v, dx, order), y, H, steps, cf)
    growth = np.linalg.norm(y) / n0
    if grows:
        assert growth > 1.5
    else:
        assert growth < 1.0 + 1e-9


def _small_acoustic(seed=11, n=12, order=4):
    y0, kappa, rho = inputs.acoustic_problem((n, n), seed, n_gauss=3, sigma=2.0)
    rng = np.random.default_rng(seed)
    y0 = y0 + 0.1 * rng.standard_normal(y0.shape)
    b = 1.0 / rho
    dx = [1.0, 1.0]
    f = lambda y, k=kappa: mol.rhs_acoustic(y, k, b, dx, order)
    fT = lambda y, k=kappa: mol.rhs_acoustic_T(y, k, b, dx, order)
    pair = lambda mu, y: mol.dA_dkappa_pairing(mu, y, dx, order)
    return y0, kappa, b, dx, f, fT, pair


def test_adjoint_dot_product_identity():
    y0, kappa, b, dx, f, fT, pair = _small_acoustic()
    _, steps, c = scheme("gbs_8_6")
    cf = W.to_fp64(c)
    H = 1.0
    rng = np.random.default_rng(1)
    w = rng.standard_normal(y0.shape)
    out = G.gbs_macro_step(f, y0, H, steps, cf)
    lam_in, _ = G.gbs_macro_step_adjoint(f, fT, pair, y0, w, H, steps, cf)
    lhs, rhs = np.sum(out * w), np.sum(y0 * lam_in)
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(out * w))


def test_adjoint_kappa_gradient_central_differences():
    y0, kappa, b, dx, _, _, _ = _small_acoustic()
    _, steps, c = SQ8
    cf = W.to_fp64(c)
    H = 0.8
    order = 4
    rng = np.random.default_rng(2)
    w = rng.standard_normal(y0.shape)

    def J(k):
        f = lambda y: mol.rhs_acoustic(y, k, b, dx, order)
        return np.sum(w * G.gbs_macro_step(f, y0, H, steps, cf))

    f = lambda y: mol.rhs_acoustic(y, kappa, b, dx, order)
    fT = lambda y: mol.rhs_acoustic_T(y, kappa, b, dx, order)
    pair = lambda mu, y: mol.dA_dkappa_pairing(mu, y, dx, order)
    _, g = G.gbs_macro_step_adjoint(f, fT, pair, y0, w, H, steps, cf)
    for _ in range(4):
        d = rng.standard_normal(kappa.shape)
        eps = 1e-5
        fd = (J(kappa + eps * d) - J(kappa - eps * d)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-7)


def test_misfit_gradient_central_differences():
    n, order = 12, 4
    y0, kappa, b, dx, _, _, _ = _small_acoustic(n=n, order=order)
    _, steps, c = SQ8
    cf = W.to_fp64(c)
    H, n_macro = 0.7, 3
    rcv = np.array([3, 17, 50, 101, 140], dtype=np.int64)
    rng = np.random.default_rng(9)
    data = rng.standard_normal((n_macro, rcv.size)) * 0.1

    def run(k):
        f = lambda y: mol.rhs_acoustic(y, k, b, dx, order)
        fT = lambda y: mol.rhs_acoustic_T(y, k, b, dx, order)
        pair = lambda mu, y: mol.dA_dkappa_pairing(mu, y, dx, order)
        return G.misfit_and_gradient(f, fT, pair, y0, H, steps, cf, n_macro, rcv, data)

    J0, g = run(kappa)
    for _ in range(3):
        d = rng.standard_normal(kappa.shape)
        eps = 1e-5
        fd = (run(kappa + eps * d)[0] - run(kappa - eps * d)[0]) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6)

