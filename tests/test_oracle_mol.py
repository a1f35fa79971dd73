"""Pins for the oracle's finite-difference operators and wave right-hand sides (no GPU).

The stencils are checked against their closed-form Fourier symbols and their
order of accuracy; the transposes against the dot-product identity; the
acoustic operator against its energy skew-symmetry (a wrong sign on any term
breaks it) and against the plane-wave symbol for constant coefficients.
"""
import numpy as np
import pytest

from oracle import mol

SYMBOL = {
    4: lambda th: (8 * np.sin(th) - np.sin(2 * th)) / 6.0,
    6: lambda th: (45 * np.sin(th) - 9 * np.sin(2 * th) + np.sin(3 * th)) / 30.0,
}


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_deriv_fourier_symbol(order, d):
    shape = (8, 12, 16)
    n = shape[2 - d]
    dx = 0.37
    rng = np.random.default_rng(order + d)
    for k in rng.integers(0, n, size=4):
        th = 2 * np.pi * k / n
        idx = np.arange(n)
        mode = np.exp(1j * th * idx)
        sh = [1, 1, 1]
        sh[2 - d] = n
        f = np.broadcast_to(mode.reshape(sh), shape).astype(np.complex128)
        got = mol.deriv(f, d, dx, order)
        expect = 1j * SYMBOL[order](th) / dx * f
        np.testing.assert_allclose(got, expect, atol=1e-12)


@pytest.mark.parametrize("order", [4, 6])
def test_deriv_order_of_accuracy(order):
    errs = []
    for n in (32, 64):
        x = 2 * np.pi * np.arange(n) / n
        f = np.sin(3 * x) + np.cos(x)
        d = mol.deriv(f, 0, 2 * np.pi / n, order)
        errs.append(np.max(np.abs(d - (3 * np.cos(3 * x) - np.sin(x)))))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.15


@pytest.mark.parametrize("order", [4, 6])
def test_deriv_transpose_identity(order):
    rng = np.random.default_rng(1)
    f = rng.standard_normal((6, 10, 14))
    g = rng.standard_normal((6, 10, 14))
    for d in range(3):
        lhs = np.sum(mol.deriv(f, d, 0.5, order) * g)
        rhs = np.sum(f * mol.deriv_T(g, d, 0.5, order))
        assert abs(lhs - rhs) < 1e-12 * np.sum(np.abs(f)) * np.sum(np.abs(g)) / f.size
        # centred stencils are antisymmetric: D^T = -D
        np.testing.assert_allclose(mol.deriv_T(g, d, 0.5, order), -mol.deriv(g, d, 0.5, order), atol=1e-12)


def _acoustic(ndim, seed=3):
    rng = np.random.default_rng(seed)
    shape = (6, 8, 10)[3 - ndim:]
    kappa = 1 + 0.5 * rng.random(shape)
    b = 1 / (1 + 0.5 * rng.random(shape))
    y = rng.standard_normal((1 + ndim,) + shape)
    dx = [0.7, 0.9, 1.1][:ndim]
    return y, kappa, b, dx


@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("order", [4, 6])
def test_acoustic_energy_skew(ndim, order):
    # <y, W A y> = 0 with W = diag(1/kappa, rho, ...): the semi-discrete energy is conserved.
    y, kappa, b, dx = _acoustic(ndim)
    f = mol.rhs_acoustic(y, kappa, b, dx, order)
    e = np.sum(y[0] * f[0] / kappa) + sum(np.sum(y[1 + d] * f[1 + d] / b) for d in range(ndim))
    scale = np.sum(np.abs(y) * np.abs(f))
    assert abs(e) < 1e-13 * scale


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("order", [4, 6])
def test_acoustic_transpose_and_kappa_pairing(ndim, order):
    y, kappa, b, dx = _acoustic(ndim)
    rng = np.random.default_rng(5)
    w = rng.standard_normal(y.shape)
    lhs = np.sum(mol.rhs_acoustic(y, kappa, b, dx, order) * w)
    rhs = np.sum(y * mol.rhs_acoustic_T(w, kappa, b, dx, order))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-12
    # A is affine in kappa: the directional derivative is exact for any step
    dk = rng.standard_normal(kappa.shape)
    a1 = np.sum(w * mol.rhs_acoustic(y, kappa + dk, b, dx, order))
    a0 = np.sum(w * mol.rhs_acoustic(y, kappa, b, dx, order))
    pair = mol.dA_dkappa_pairing(w, y, dx, order)
    assert abs((a1 - a0) - np.sum(pair * dk)) < 1e-11 * (abs(a1) + abs(a0))


def test_wave1d_transpose():
    rng = np.random.default_rng(2)
    y = rng.standard_normal((2, 33))
    w = rng.standard_normal((2, 33))
    for order in (4, 6):
        lhs = np.sum(mol.rhs_wave1d(y, 0.3, order) * w)
        rhs = np.sum(y * mol.rhs_wave1d_T(w, 0.3, order))
        assert abs(lhs - rhs) < 1e-12


@pytest.mark.parametrize("order", [4, 6])
def test_constant_coefficient_plane_wave_eigenvalues(order):
    # For constant kappa, b the 2D operator on mode (kx, ky) has eigenvalues 0 and
    # +-i c sqrt(sx^2 + sy^2), c = sqrt(kappa b), s = symbol/dx.
    n, kappa0, b0, dx = 16, 2.0, 0.5, [1.0, 1.0]
    kappa = np.full((n, n), kappa0)
    b = np.full((n, n), b0)
    th = 2 * np.pi * np.arange(n) / n
    smax = 0.0
    for kx in range(n):
        for ky in range(n):
            sx, sy = SYMBOL[order](th[kx]), SYMBOL[order](th[ky])
            smax = max(smax, np.sqrt(kappa0 * b0) * np.hypot(sx, sy))
    rho = mol.power_iteration_rho(lambda v: mol.rhs_acoustic(v, kappa, b, dx, order), (3, n, n), iters=400)
    assert rho == pytest.approx(smax, rel=1e-6)


def test_symbol_max_values():
    # max |symbol| x dx of the centred stencils: 4th order ~1.3722, 6th order ~1.5860
    for order, expect in ((4, 1.3722), (6, 1.5860)):
        th = np.linspace(0, np.pi, 100001)
        assert mol.symbol_max(order) == pytest.approx(np.max(np.abs(SYMBOL[order](th))), rel=1e-8)
        assert round(mol.symbol_max(order), 4) == expect
