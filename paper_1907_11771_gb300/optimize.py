"""Imaginary-axis stability optimisation of extrapolation weights (App. B).

Given an even order p and step counts n_1..n_m (m > p/2), find free weights
c_free that maximise the time step h such that |R(h lambda)| <= 1 on the
contour lambda in [0, i] (the stretch [-i, 0] follows by symmetry, the
coefficients being real), subject to the order constraints V c = b
(Sec. 3.2 eq. "vander") -- App. B eqs. "problem1" and "reformulated_problem":
a bisection over h around the convex minimax subproblem (eq. "cvx_subproblem")

    r(h) = min over c_free of  max over the contour of |R(h lambda)| - 1.

The order constraints are kept exact by eliminating the dependent weights,
c_dep = V_dep^-1 (b - V_free c_free) (Sec. 3.7 eq. "cdep_computation"), so R
is affine in c_free.  The value of the subproblem
is never below zero (|R(0)| = 1), so its optimal set is degenerate; what the
bisection needs is feasibility -- some c_free with |R|^2 <= 1 + tol on every
sample of the contour -- which is decided by minimising the convex penalty
sum_j max(0, |R_j|^2 - 1)^2 (L-BFGS on scaled variables).  One more linear constraint keeps the
stability region open along the axis near the origin: with R(xi) = e^xi +
e_(p+1) xi^(p+1) + e_(p+2) xi^(p+2) + ..., |R(iy)|^2 - 1 starts with
2 s (e_(p+1) - e_(p+2)) y^(p+2), s = +1 for p = 0 mod 4 and -1 for p = 2 mod 4,
which must be negative (the sign of a_(p+2) in Sec. 3.5).

Stability polynomials are evaluated through the GBS recurrence on the test
equation (well conditioned on the imaginary axis for |h lambda| <= N_k).
This is a host-side design tool: it produces weights for gbs_set_weights and is
checked by exact root isolation of the resulting R.
"""
from dataclasses import dataclass
from fractions import Fraction
from math import factorial

import numpy as np
from scipy.optimize import minimize


def _vandermonde(steps, order):
    return [[Fraction(1, n) ** (2 * j) for n in steps] for j in range(order // 2)]


def _solve(A, b):
    n = len(A)
    M = [list(map(Fraction, A[i])) + [Fraction(b[i])] for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        p = M[col][col]
        M[col] = [v / p for v in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
    return [M[i][n] for i in range(n)]


def affine_weights(order, steps_dep, steps_free):
    """c = c0 + G c_free with c = (c_dep, c_free): exact rational c0 (|dep|+|free|) and G."""
    q = order // 2
    Vd = _vandermonde(steps_dep, order)
    Vf = _vandermonde(steps_free, order)
    b = [Fraction(1)] + [Fraction(0)] * (q - 1)
    c_dep0 = _solve(Vd, b)
    cols = []
    for f in range(len(steps_free)):
        cols.append(_solve(Vd, [-Vf[j][f] for j in range(q)]))
    m = len(steps_dep) + len(steps_free)
    c0 = np.zeros(m)
    G = np.zeros((m, len(steps_free)))
    c0[:q] = [float(v) for v in c_dep0]
    for f, col in enumerate(cols):
        G[:q, f] = [float(v) for v in col]
        G[q + f, f] = 1.0
    return c0, G


def gbs_poly_values(n, xi):
    """P_n(xi) for an array of complex xi via the GBS recurrence (FE, n LF steps, averaging)."""
    z = xi / n
    ym, yc = np.ones_like(xi), 1.0 + z
    before = ym
    for _ in range(n):
        yn = ym + 2.0 * z * yc
        before, ym, yc = ym, yc, yn
    return (before + 2.0 * ym + yc) / 4.0


def gbs_poly_coeffs(n, upto):
    """Taylor coefficients of P_n up to degree ``upto`` (exact rationals)."""
    zf = Fraction(1, n)
    ys = [[Fraction(1)]]
    ys.append([Fraction(1), zf])

    def add(a, b):
        k = max(len(a), len(b))
        return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(k)]

    for j in range(1, n + 1):
        ys.append(add(ys[j - 1], [Fraction(0)] + [2 * zf * v for v in ys[j]]))
    P = add(add(ys[n - 1], [2 * v for v in ys[n]]), ys[n + 1])
    P = [v / 4 for v in P]
    return [P[k] if k < len(P) else Fraction(0) for k in range(upto + 1)]


@dataclass
class OptResult:
    steps_dep: tuple
    steps_free: tuple
    c_free: np.ndarray
    isb: float          # the bisection's h (ISB of the optimised scheme, up to the LP tolerance)
    isb_n: float        # isb / (N_max + 1)


def _solve_samples(h, steps, c0, G, lead, x0, ys, margin, order, penalty_scale=1e10):
    """For fixed h, minimise sum_j max(0, |R(i h y_j)|^2 - 1 + m_j)^2 (+ the lead-term hinge)
    over the free weights: convex and once differentiable (each |R_j|^2 is a convex
    quadratic of the affine R_j).  Returns the weights."""
    xi = 1j * h * ys
    P = np.stack([gbs_poly_values(n, xi) for n in steps], axis=1)     # samples x m
    Q0, QG = P @ c0, P @ G
    m = _margin(h, ys, margin, order)
    D = 1.0 / np.maximum(np.linalg.norm(QG, axis=0), 1e-300)         # variable scaling x = D z
    QGs = QG * D[None, :]
    la, lb = lead
    la_s = la * D

    def f(z):
        R = Q0 + QGs @ z
        v = np.maximum(R.real ** 2 + R.imag ** 2 - 1.0 + m, 0.0) * penalty_scale
        lv = max(la_s @ z + lb, 0.0) * penalty_scale
        dg = 2.0 * (R.real[:, None] * QGs.real + R.imag[:, None] * QGs.imag)
        return float(np.sum(v * v) + lv * lv), 2.0 * penalty_scale * ((v[:, None] * dg).sum(0) + lv * la_s)

    res = minimize(f, np.asarray(x0, float) / D, jac=True, method="L-BFGS-B",
                   options={"maxiter": 20000, "ftol": 1e-32, "gtol": 1e-32, "maxcor": 30})
    return res.x * D


def _margin(h, ys, margin, order):
    # a margin inside the unit circle, vanishing like |h y|^(p+2) at the origin where the
    # lead-term constraint takes over
    return margin * np.minimum(1.0, (h * ys / 4.0) ** (order + 2))


def _violations(h, steps, c0, G, lead, x, ys, margin, order):
    xi = 1j * h * ys
    P = np.stack([gbs_poly_values(n, xi) for n in steps], axis=1)
    R = P @ (c0 + G @ x)
    return R.real ** 2 + R.imag ** 2 - 1.0 + _margin(h, ys, margin, order), float(lead[0] @ x + lead[1])


def _feasible_weights(h, steps, c0, G, lead, x0, ys, margin, order, tol, refine=20, rounds=8):
    """Exchange method: solve on the sample set, check a grid `refine` times finer, add the
    points (and their neighbours) where |R| leaves the margin, repeat.  Returns (worst, x)."""
    fine = np.arange(1, refine * ys.size + 1) / (refine * ys.size)
    pts = ys.copy()
    x = np.asarray(x0, float)
    worst = np.inf
    for _ in range(rounds):
        x = _solve_samples(h, steps, c0, G, lead, x, pts, margin, order)
        v, lv = _violations(h, steps, c0, G, lead, x, fine, margin, order)
        worst = max(float(v.max()), lv)
        if worst <= tol:
            return worst, x
        bad = np.where(v > tol)[0]
        if bad.size == 0:
            return worst, x
        add = np.unique(np.clip(np.concatenate([bad - 1, bad, bad + 1]), 0, fine.size - 1))
        pts = np.unique(np.concatenate([pts, fine[add]]))
    return worst, x


def optimise(order, steps_dep, steps_free, h_lo, h_hi=None, n_samples=600, iters=30, tol=1e-13,
             x0=None, lead_margin=1e-14, margin=1e-8):
    """Maximise the imaginary stability boundary over the free weights (App. B).

    Bisection over h; at each h the convex subproblem is solved as a smooth penalty
    minimisation (the minimax of eq. "cvx_subproblem" is degenerate because |R(0)| = 1, so
    feasibility -- every sample with |R|^2 <= 1 + tol and the lead-term sign respected -- is
    the test).  h_lo must be feasible (e.g. a fraction of a known scheme's ISB)."""
    steps_dep, steps_free = tuple(steps_dep), tuple(steps_free)
    steps = steps_dep + steps_free
    c0, G = affine_weights(order, steps_dep, steps_free)
    nmax = max(steps)
    coef = np.array([[float(v) for v in gbs_poly_coeffs(n, order + 2)] for n in steps])   # m x (p+3)
    ek = lambda k: (coef[:, k] @ G, coef[:, k] @ c0 - 1.0 / factorial(k))
    g1, r1 = ek(order + 1)
    g2, r2 = ek(order + 2)
    sg = 1.0 if order % 4 == 0 else -1.0
    # |R(iy)|^2 - 1 = 2 sg (e_(p+1) - e_(p+2)) y^(p+2) + ...: keep it negative
    lscale = 1.0 / max(np.max(np.abs(g1 - g2)), 1e-300)
    lead = (2 * sg * (g1 - g2) * lscale, (2 * sg * (r1 - r2) + lead_margin) * lscale)
    ys = np.arange(1, n_samples + 1) / n_samples
    hi = h_hi if h_hi is not None else float(nmax + 1)
    x = np.zeros(len(steps_free)) if x0 is None else np.asarray(x0, float)
    worst, x = _feasible_weights(h_lo, steps, c0, G, lead, x, ys, margin, order, tol)
    if worst > tol:
        raise ValueError(f"h_lo = {h_lo} is not feasible (violation {worst:.2e})")
    lo, best = h_lo, x
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        worst, xm = _feasible_weights(mid, steps, c0, G, lead, best, ys, margin, order, tol)
        if worst <= tol:
            lo, best = mid, xm
        else:
            hi = mid
        if hi - lo < 1e-6 * hi:
            break
    return OptResult(steps_dep, steps_free, best, lo, lo / (nmax + 1))


def rationalize(values, max_den=1 << 20):
    """Nearby small rationals for the free weights (the paper prints such rationals, Sec. 3.8)."""
    return [Fraction(float(v)).limit_denominator(max_den) for v in values]
