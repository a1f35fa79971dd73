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
is affine in c_free.  Since |R(0)| = 1 the subproblem's value is never below
zero; the bisection needs its feasibility at a given h, decided here by linear
programming on samples y_j of the contour:

* |R_j| <= 1 - mu_j is the intersection of the half-planes
  Re(e^(-i phi) R_j) <= 1 - mu_j over all phi.  The LP starts from eight
  angles per sample and adds the tangent cut at phi = arg R_j wherever the
  solution still leaves the circle (cutting planes), until every sample holds
  to 1e-13.  mu_j = margin min(1, (h y_j / 4)^(p+2)) keeps the solution off the
  circle away from the origin.
* Near the origin the free weights move R only at O(y^(p+1)) (the order
  constraints), below rounding: samples where they cannot move R by 1e-8 of
  their largest effect are left to one linear constraint that keeps the
  stability region open along the axis.  With R(xi) = e^xi + e_(p+1) xi^(p+1)
  + e_(p+2) xi^(p+2) + ..., |R(iy)|^2 - 1 starts with
  2 s (e_(p+1) - e_(p+2)) y^(p+2), s = +1 for p = 0 mod 4 and -1 for
  p = 2 mod 4, which must be negative (the sign of a_(p+2) in Sec. 3.5); its
  margin is relative, since these coefficients scale like 1/(p+1)!.
* The LP's objective is a margin t weighted by each sample's sensitivity to
  the free weights, which makes the LP always feasible and picks a central
  point; h is feasible when the cut loop converges.
* Exchange: the solution is checked on a grid `refine` times finer, points
  that leave the circle (by more than half the margin) join the samples, and
  the LP is solved again.
* Every LP is centred on the weights of the largest feasible h so far, which
  keeps its right-hand sides moderate.

Stability polynomials are evaluated through the GBS recurrence on the test
equation (well conditioned on the imaginary axis for |h lambda| <= N_k).
This is a host-side design tool: it produces weights for gbs_set_weights and is
checked by exact root isolation of the resulting R.  For order 8 on all even
counts up to 22 and up to 30, and order 4 up to 28, it reproduces the optimal
ISB_n the paper prints (Sec. 3.8, Table 2); at order 12 and 16 the LP's
tolerances no longer resolve the constraints (rows whose sensitivities span
many decades) and it stops short of the printed optima.
"""
from dataclasses import dataclass
from fractions import Fraction
from math import factorial

import numpy as np
from scipy.optimize import linprog


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
    isb: float          # the bisection's h (ISB of the optimised scheme, up to the sampling)
    isb_n: float        # isb / (N_max + 1)


def _lead_constraint(order, steps, c0, G):
    """(g, r): 2 s (e_(p+1) - e_(p+2)) = g . c_free + r, the leading term of |R(iy)|^2 - 1."""
    coef = np.array([[float(v) for v in gbs_poly_coeffs(n, order + 2)] for n in steps])   # m x (p+3)
    ek = lambda k: (coef[:, k] @ G, coef[:, k] @ c0 - 1.0 / factorial(k))
    g1, r1 = ek(order + 1)
    g2, r2 = ek(order + 2)
    sg = 1.0 if order % 4 == 0 else -1.0
    return 2 * sg * (g1 - g2), 2 * sg * (r1 - r2)


def _margin(h, ys, margin, order):
    # a margin inside the unit circle, vanishing like |h y|^(p+2) at the origin where the
    # lead-term constraint takes over
    return margin * np.minimum(1.0, (h * ys / 4.0) ** (order + 2))


def _lp_feasible(h, steps, c0, G, lead, order, ys, margin, x0, tol=1e-13, angles=8, rounds=40):
    """Free weights with |R(i h y_j)| <= 1 - mu_j on the samples and the lead term negative,
    by cutting planes around x0; None if the LP proves none exists or the cuts do not settle."""
    P = np.stack([gbs_poly_values(n, 1j * h * ys) for n in steps], axis=1)
    a, B = P @ (c0 + G @ x0), P @ G
    D = 1.0 / np.maximum(np.abs(B).max(axis=0), 1e-300)     # column scaling: x = x0 + D z
    Bs = B * D[None, :]
    sens = np.abs(Bs).max(axis=1)
    keep = sens > 1e-8
    a, Bs, sens = a[keep], Bs[keep], sens[keep]
    mu = _margin(h, ys[keep], margin, order)
    nf = G.shape[1]
    rows, rhs = [], []

    def cut(j, phi):
        e = np.exp(-1j * phi)
        r = (e * Bs[j]).real
        sc = 1.0 / max(np.abs(r).max(), sens[j])
        rows.append(np.concatenate([r * sc, [-sens[j] * sc]]))
        rhs.append((1.0 - mu[j] - (e * a[j]).real) * sc)

    for j in range(a.size):
        for k in range(angles):
            cut(j, 2 * np.pi * k / angles)
    lg, lr = lead
    eps = 1e-8 * abs(lr)
    ls = 1.0 / max(np.abs(lg * D).max(), 1e-300)
    lead_row = np.concatenate([lg * D * ls, [0.0]])
    lead_rhs = -(lr + lg @ x0 + eps) * ls
    cost = np.zeros(nf + 1)
    cost[-1] = 1.0
    bounds = [(None, None)] * nf + [(-1.0, None)]
    for _ in range(rounds):
        A_ub, b_ub = np.array(rows + [lead_row]), np.array(rhs + [lead_rhs])
        res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs-ds")
        if res.status == 4:   # numerical trouble in the simplex: try the interior-point method
            res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs-ipm")
        if res.status != 0 or res.x[-1] > 0:
            return None
        z = res.x[:nf]
        R = a + Bs @ z
        v = np.abs(R) - 1 + mu
        if v.max() <= tol:
            return x0 + z * D
        for j in np.where(v > tol)[0]:
            cut(j, np.angle(R[j]))
    return None


def _feasible(h, steps, c0, G, lead, order, ys, fine, margin, x0, tol=1e-13, rounds=6):
    """Exchange loop around the LP: weights stable on the fine grid (half the margin), or None."""
    pts = ys
    for _ in range(rounds):
        x = _lp_feasible(h, steps, c0, G, lead, order, pts, margin, x0)
        if x is None:
            return None
        P = np.stack([gbs_poly_values(n, 1j * h * fine) for n in steps], axis=1)
        v = np.abs(P @ (c0 + G @ x)) - 1 + 0.5 * _margin(h, fine, margin, order)
        bad = np.where(v > tol)[0]
        if bad.size == 0:
            return x
        pts = np.unique(np.concatenate([pts, fine[bad]]))
    return None


def optimise(order, steps_dep, steps_free, n_samples=600, refine=60, margin=1e-7, rel_tol=1e-7, h_hi=None):
    """Maximise the imaginary stability boundary over the free weights (App. B): bisection over
    h in (0, N_max + 1] with the LP feasibility test above.  The dependent/free split only fixes
    the parametrisation (every split spans the same weights); small dependent counts keep it
    well conditioned."""
    steps_dep, steps_free = tuple(steps_dep), tuple(steps_free)
    steps = steps_dep + steps_free
    c0, G = affine_weights(order, steps_dep, steps_free)
    lead = _lead_constraint(order, steps, c0, G)
    nmax = max(steps)
    ys = np.arange(1, n_samples + 1) / n_samples
    fine = np.arange(1, refine * n_samples + 1) / (refine * n_samples)
    lo, hi = 0.0, float(h_hi if h_hi is not None else nmax + 1)
    best = np.zeros(len(steps_free))
    found = False
    while hi - lo > rel_tol * hi:
        mid = 0.5 * (lo + hi)
        x = _feasible(mid, steps, c0, G, lead, order, ys, fine, margin, best)
        if x is not None:
            lo, best, found = mid, x, True
        else:
            hi = mid
    if not found:
        raise ValueError("no stable free weights found")
    return OptResult(steps_dep, steps_free, best, lo, lo / (nmax + 1))


def rationalize(values, max_den=1 << 20):
    """Nearby small rationals for the free weights (the paper prints such rationals, Sec. 3.8)."""
    return [Fraction(float(v)).limit_denominator(max_den) for v in values]
