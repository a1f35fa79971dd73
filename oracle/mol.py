"""Method-of-lines right-hand sides y' = f(y) = A y (oracle side, FP64 by default).

The paper fixes only the ODE solver; the spatial operators are the wave
systems of the workloads this library targets (Appendix A.1: for wave-type
PDEs the eigenvalues of the spatial operator lie along the imaginary axis, so
the solver's imaginary stability boundary sets the time step).  All operators
are periodic, collocated, centred finite differences, written as plain sums of
shifted copies (``numpy.roll``):

* order 4:  f'(x) ~ [f(x-2h) - 8 f(x-h) + 8 f(x+h) - f(x+2h)] / (12 h)
* order 6:  f'(x) ~ [-f(x-3h) + 9 f(x-2h) - 45 f(x-h) + 45 f(x+h) - 9 f(x+2h) + f(x+3h)] / (60 h)

Array layout: a state is an array ``y[field, (z,) (y,) x]`` with x the last
(fastest) axis.  Spatial direction d = 0, 1, 2 means x, y, z, i.e. array axis
``-1 - d`` of a field.

Systems
* 1D wave:   u_t = v_x, v_t = u_x                  fields (u, v)
* acoustics: p_t = -kappa div(u), u_d,t = -b d_d p  fields (p, u_x, u_y[, u_z]),
  b = 1/rho.
* one-way wave with a spectral derivative (Sec. 4): u_t = -u_x, field (u), the derivative
  taken exactly on every resolved Fourier mode (FFT, multiply by i k, inverse FFT; the Nyquist
  mode, whose derivative the grid cannot represent, is set to zero).

The transposes (used by the discrete adjoint) are formed literally: the
transpose of "shift by +j" is "shift by -j"; no antisymmetry is assumed.
"""
from fractions import Fraction

import numpy as np

# offset j -> weight w_j, derivative = sum_j w_j f(x + j dx) / dx
FD_WEIGHTS = {
    4: {-2: Fraction(1, 12), -1: Fraction(-8, 12), 1: Fraction(8, 12), 2: Fraction(-1, 12)},
    6: {-3: Fraction(-1, 60), -2: Fraction(9, 60), -1: Fraction(-45, 60),
        1: Fraction(45, 60), 2: Fraction(-9, 60), 3: Fraction(1, 60)},
}


def _axis(f, d):
    return f.ndim - 1 - d


def deriv(f, d, dx, order):
    """Centred periodic first derivative of the field ``f`` along direction d.
    Textbook 4th/6th-order weights; the paper fixes no spatial operator (Sec. 4 uses spectral ones)."""
    dt = f.dtype.type
    out = np.zeros_like(f)
    for j, w in FD_WEIGHTS[order].items():
        out = out + dt(float(w)) * np.roll(f, -j, axis=_axis(f, d))
    return out / dt(dx)


def deriv_T(f, d, dx, order):
    """Transpose of ``deriv`` (each shift replaced by the opposite shift); for the adjoint, not in the paper."""
    dt = f.dtype.type
    out = np.zeros_like(f)
    for j, w in FD_WEIGHTS[order].items():
        out = out + dt(float(w)) * np.roll(f, j, axis=_axis(f, d))
    return out / dt(dx)


# --------------------------------------------------------------------------
# 1D wave system u_t = v_x, v_t = u_x
# --------------------------------------------------------------------------

def rhs_wave1d(y, dx, order):
    u, v = y
    return np.stack([deriv(v, 0, dx, order), deriv(u, 0, dx, order)])


def rhs_wave1d_T(lam, dx, order):
    lu, lv = lam
    return np.stack([deriv_T(lv, 0, dx, order), deriv_T(lu, 0, dx, order)])


# --------------------------------------------------------------------------
# Acoustics p_t = -kappa div u, u_d,t = -b d_d p  (d-dimensional)
# --------------------------------------------------------------------------

def rhs_acoustic(y, kappa, b, dx, order):
    """f(y) for y = (p, u_x, u_y[, u_z]); kappa, b arrays of the grid shape.
    The right-hand side of y' = f(y) (Sec. 2.1) for linear acoustics; the paper fixes no system."""
    ndim = y.ndim - 1
    p = y[0]
    div = np.zeros_like(p)
    for d in range(ndim):
        div = div + deriv(y[1 + d], d, dx[d], order)
    out = [-(kappa * div)]
    for d in range(ndim):
        out.append(-(b * deriv(p, d, dx[d], order)))
    return np.stack(out)


def rhs_acoustic_T(lam, kappa, b, dx, order):
    """A^T lam for the acoustic operator A(kappa, b) of ``rhs_acoustic`` (adjoint; not in the paper)."""
    ndim = lam.ndim - 1
    lp = lam[0]
    out_p = np.zeros_like(lp)
    for d in range(ndim):
        out_p = out_p + deriv_T(-(b * lam[1 + d]), d, dx[d], order)
    out = [out_p]
    for d in range(ndim):
        out.append(deriv_T(-(kappa * lp), d, dx[d], order))
    return np.stack(out)


def dA_dkappa_pairing(mu, y, dx, order):
    """Not in the paper (gradient with respect to kappa).
    Pointwise <mu, (dA/dkappa_i) y>: the p row of A y is -kappa div u, so the
    derivative with respect to kappa at point i is mu_p[i] * (-div u)[i]."""
    ndim = y.ndim - 1
    div = np.zeros_like(y[0])
    for d in range(ndim):
        div = div + deriv(y[1 + d], d, dx[d], order)
    return mu[0] * (-div)


# --------------------------------------------------------------------------
# Spectral information
def rhs_oneway_spectral(y, dx):
    """f(u) = -u_x for u_t + u_x = 0 on a periodic grid of n points, spacing dx (Sec. 4).

    Mode m of the discrete Fourier transform (m = -n/2+1 .. n/2-1) has wavenumber
    k = 2 pi m / (n dx) and derivative i k; the Nyquist mode m = n/2 gets 0."""
    n = y.shape[-1]
    m = np.fft.fftfreq(n, d=1.0 / n)              # 0, 1, .., n/2-1, -n/2, .., -1
    k = 2.0 * np.pi * m / (n * dx)
    if n % 2 == 0:
        k[n // 2] = 0.0
    return -np.real(np.fft.ifft(1j * k * np.fft.fft(y, axis=-1), axis=-1))


# --------------------------------------------------------------------------

def symbol_max(order):
    """max over theta of |sum_j w_j sin(j theta)|, the largest |symbol| x dx of ``deriv``
    (found by dense sampling plus a local refinement; used only for step sizes)."""
    th = np.linspace(0.0, np.pi, 200001)
    s = sum(float(w) * np.sin(j * th) for j, w in FD_WEIGHTS[order].items())
    i = int(np.argmax(np.abs(s)))
    lo, hi = th[max(i - 1, 0)], th[min(i + 1, th.size - 1)]
    for _ in range(100):
        m1, m2 = lo + (hi - lo) / 3, hi - (hi - lo) / 3
        f = lambda t: abs(sum(float(w) * np.sin(j * t) for j, w in FD_WEIGHTS[order].items()))
        if f(m1) < f(m2):
            lo = m1
        else:
            hi = m2
    t = (lo + hi) / 2
    return abs(sum(float(w) * np.sin(j * t) for j, w in FD_WEIGHTS[order].items()))


def power_iteration_rho(apply_A, y_shape, iters=300, seed=0):
    """Estimate the spectral radius of A by power iteration on A^2: the bound on |lambda| that
    App. A.1 scales by the step to place the spectrum in the stability domain.

    For the operators here A is skew-adjoint in an energy inner product, so its
    eigenvalues are +-i omega and A^2 has the real, non-positive eigenvalues
    -omega^2; the iteration on A^2 converges to the largest omega^2."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(y_shape)
    x /= np.linalg.norm(x)
    lam2 = 0.0
    for _ in range(iters):
        z = apply_A(apply_A(x))
        lam2 = np.linalg.norm(z)
        x = z / lam2
    return float(np.sqrt(lam2))
