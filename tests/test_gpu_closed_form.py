"""GPU macro-steps against the closed form for constant coefficients (no oracle time stepping).

For constant kappa and b on a periodic grid the semi-discrete acoustic operator is diagonal in
Fourier space: mode k evolves by the F x F symbol matrix A_k (entries -i kappa s_d and
-i b s_d, s_d the centred-difference symbol along axis d).  A GBS macro-step of size H is a
polynomial in H A, the scheme's stability polynomial R (Sec. 2.1, Appendix A), so each mode is
multiplied by the matrix R(H A_k).  M macro-steps give R(H A_k)^M.  This checks every CUDA path
(FP64, FP32 pairs, FP32 plain, the time-blocked FP32 kernel) against that product; R's
coefficients are the exact rationals of the scheme's weights.

Tolerances (relative L2 over the state): FP64 1e-12 and pairs 1e-10 as in the other parity
tests.  FP32 states: each y*_k carries at most about (N_k + 1) FP32 roundings of |y| (one per
Forward-Euler or leap-frog update; the leap-frog recursion does not amplify them below the
stability limit) and the combine weights them by |c_k|, so the bound is
n_macro 2^-24 sum_k |c_k| (N_k + 1): 4.0e-5 per macro-step for GBS_8,6.  The inputs are white
noise, so every wavenumber up to the grid's Nyquist mode is exercised.
"""
import decimal
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import weights as OW
from paper_1907_11771_gb300 import binding as B
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300.solver import GBSSolver
from tests.gpu_common import GOLD, GOLD_OF, rel_l2

pytestmark = pytest.mark.gpu
F64, X2, F32 = B.GBS_F64, B.GBS_F32X2, B.GBS_F32_STATE_F64_COMBINE
TOL = {F64: 1e-12, X2: 1e-10}
KAPPA0, RHO0 = 1.5, 0.5            # b = 1 / rho = 2, exact in every precision


def symbol(order, th):
    """i s(theta) dx is the Fourier symbol of the centred first-derivative stencil."""
    if order == 4:
        return (8 * np.sin(th) - np.sin(2 * th)) / 6
    return (45 * np.sin(th) - 9 * np.sin(2 * th) + np.sin(3 * th)) / 30


def exact_scheme(scheme):
    g = GOLD[GOLD_OF[scheme.name]]
    dep = [int(t) for t in g["dep"].split()]
    free = [int(t) for t in g.get("free", "").split()]
    cf = [Fraction(t) for t in g.get("cfree", "").split()]
    return OW.scheme_weights(int(g["order"]), dep, free, cf)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_11771_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def closed_form(y0, order, H, n_macro, scheme):
    """y after n_macro macro-steps: mode by mode R(H A_k)^n_macro y0_k.

    A_k = [[0, -i kappa s^T], [-i b s, 0]] satisfies A^3 = -w^2 A with w^2 = kappa b |s|^2, so
    R(H A) = a_0 I + alpha A + beta A^2 with alpha = sum_m a_(2m+1) H^(2m+1) (-w^2)^m and
    beta = sum_m a_(2m+2) H^(2m+2) (-w^2)^m.  Near the stability limit (|H w| up to about 14)
    these sums cancel terms of order 1e5 down to order 1, so they are evaluated in 50-digit
    decimal arithmetic from the exact coefficients; everything else is FP64."""
    steps, c = exact_scheme(scheme)
    R = OW.stability_poly(steps, c)                     # exact rationals a_0 .. a_deg
    F, shape = y0.shape[0], y0.shape[1:]
    nd = len(shape)
    axes = tuple(range(1, nd + 1))
    Y = np.fft.fftn(y0, axes=axes)
    grids = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(n) for n in shape], indexing="ij")
    s = [symbol(order, g) for g in grids]               # spatial axes in (z,) y, x order
    s = s[::-1]                                          # s[0] along x, s[1] along y, s[2] along z
    b0 = 1.0 / RHO0
    A = np.zeros(shape + (F, F), complex)
    for d in range(nd):
        A[..., 0, 1 + d] = -KAPPA0 * 1j * s[d]
        A[..., 1 + d, 0] = -b0 * 1j * s[d]
    w2 = KAPPA0 * b0 * sum(sd * sd for sd in s)
    with decimal.localcontext() as ctx:
        ctx.prec = 50
        a = [decimal.Decimal(q.numerator) / decimal.Decimal(q.denominator) for q in R]
        Hd = decimal.Decimal(H)
        alpha, beta = np.empty(w2.shape), np.empty(w2.shape)
        cache = {}
        for idx, v in np.ndenumerate(w2):
            if v not in cache:
                x = -decimal.Decimal(float(v)) * Hd * Hd     # (-w^2 H^2)
                al, be, pw = decimal.Decimal(0), decimal.Decimal(0), decimal.Decimal(1)
                for m in range((len(a) + 1) // 2):
                    if 2 * m + 1 < len(a):
                        al += a[2 * m + 1] * pw
                    if 2 * m + 2 < len(a):
                        be += a[2 * m + 2] * pw
                    pw *= x
                cache[v] = (float(al * Hd), float(be * Hd * Hd))
            alpha[idx], beta[idx] = cache[v]
    eye = np.broadcast_to(np.eye(F, dtype=complex), A.shape)
    M = float(R[0]) * eye + alpha[..., None, None] * A + beta[..., None, None] * (A @ A)
    Yk = np.moveaxis(Y, 0, -1)[..., None]              # (..., F, 1)
    for _ in range(n_macro):
        Yk = M @ Yk
    out = np.fft.ifftn(np.moveaxis(Yk[..., 0], -1, 0), axes=axes)
    assert np.abs(out.imag).max() <= 1e-12 * np.abs(out.real).max()
    return out.real


def tolerance(prec, scheme, n_macro):
    if prec != F32:
        return TOL[prec]
    steps, c = exact_scheme(scheme)
    return n_macro * 2.0 ** -24 * sum(abs(float(ck)) * (n + 1) for ck, n in zip(c, steps))


def gpu_run(shape_zyx, order, prec, kernel, scheme, n_macro, seed):
    rng = np.random.default_rng(seed)
    nd = len(shape_zyx)
    y0 = rng.standard_normal((1 + nd,) + tuple(shape_zyx))
    npdt = np.float32 if prec == F32 else np.float64
    y0 = y0.astype(npdt).astype(np.float64)
    dt = torch.float32 if prec == F32 else torch.float64
    pts = int(np.prod(shape_zyx))
    kappa = torch.full((pts,), KAPPA0, dtype=dt, device="cuda")
    rho = torch.full((pts,), RHO0, dtype=dt, device="cuda")
    sol = GBSSolver(B.GBS_ACOUSTIC, [tuple(reversed(shape_zyx))], [(1.0,) * nd], fd_order=order, precision=prec,
                    kappa=kappa, rho=rho)
    sol.set_scheme(scheme)
    if kernel is not None:
        sol.set_option("kernel", kernel)
    H = 0.8 * sol.stability_limit()[0]
    y = torch.tensor(y0.ravel(), dtype=dt, device="cuda")
    out = torch.empty_like(y)
    sol.step(y, out, H, n_macro)
    sol.sync()
    fused = sol.uses_fused()
    g = out.cpu().numpy().astype(np.float64).reshape(y0.shape)
    sol.close()
    return y0, g, H, fused


@pytest.mark.parametrize("order", [4, 6])
@pytest.mark.parametrize("prec,kernel", [(F64, B.GBS_KERNEL_PLAIN), (X2, B.GBS_KERNEL_PLAIN), (X2, B.GBS_KERNEL_FUSED),
                                         (F32, B.GBS_KERNEL_PLAIN), (F32, B.GBS_KERNEL_FUSED)])
def test_acoustic2d_modes_follow_matrix_R(order, prec, kernel):
    shape = (40, 72)                      # ragged against the 32 x 32 tiles in both directions
    y0, g, H, fused = gpu_run(shape, order, prec, kernel, S.GBS_8_6, 3, seed=7)
    assert fused == (kernel == B.GBS_KERNEL_FUSED)
    err = rel_l2(g, closed_form(y0, order, H, 3, S.GBS_8_6))
    assert err <= tolerance(prec, S.GBS_8_6, 3), err


@pytest.mark.parametrize("prec", [F64, X2, F32])
def test_acoustic3d_modes_follow_matrix_R(prec):
    shape = (12, 20, 36)
    y0, g, H, _ = gpu_run(shape, 4, prec, None, S.GBS_8_6, 2, seed=8)
    err = rel_l2(g, closed_form(y0, 4, H, 2, S.GBS_8_6))
    assert err <= tolerance(prec, S.GBS_8_6, 2), err
