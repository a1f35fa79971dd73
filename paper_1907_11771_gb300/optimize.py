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

* The unknown is delta(xi) = e^(-xi) R(xi) - 1 rather than R: |R| <= 1 is
  |1 + delta| <= 1, and delta, O(xi^(p+1)) near the origin, is computed
  without cancelling against 1 -- from the exact Taylor coefficients of
  R - e^xi (rational arithmetic on the GBS polynomials, whose first p + 1
  vanish by the order constraints) for |xi| <= 6, from the GBS recurrence on
  the test equation further out.  So every sample keeps its relative accuracy,
  however little the free weights move it.
* |1 + delta_j| <= 1 - mu_j is the intersection of the half-planes
  Re(e^(-i psi) delta_j) <= 1 - cos psi - mu_j over all psi.  The LP starts
  from eight angles per sample and adds the tangent cut at psi = arg(1 + delta_j)
  wherever the solution still leaves the circle (cutting planes), until every
  sample's excess is below 1e-10 of its sensitivity to the free weights.
  mu_j = margin min(1, (h y_j / 4)^(p+2)) keeps the solution off the circle
  away from the origin.
* One linear constraint keeps the stability region open along the axis at the
  origin: with R(xi) = e^xi + e_(p+1) xi^(p+1) + e_(p+2) xi^(p+2) + ...,
  |R(iy)|^2 - 1 starts with 2 s (e_(p+1) - e_(p+2)) y^(p+2), s = +1 for
  p = 0 mod 4 and -1 for p = 2 mod 4, which must be negative (the sign of
  a_(p+2) in Sec. 3.5); its margin is relative, since these coefficients scale
  like 1/(p+1)!.
* The LP's objective is a margin t weighted by each sample's sensitivity,
  which makes the LP always feasible and picks a central point; h is feasible
  when the cut loop converges with t <= 0.
* Exchange: the solution is checked on a grid `refine` times finer, points
  that leave the circle (by more than half the margin) join the samples, and
  the LP is solved again.
* Every LP is centred on the weights of the largest feasible h so far, with the
  free weights scaled column by column, which keeps its entries moderate.

* Continuation (optional): after the bisection, h rises in small steps, each
  test centred on the last feasible weights, and a step is kept only if |R| - 1
  stays within the slack on the fine grid refined around its local maxima.

This is a host-side design tool: it produces weights for gbs_set_weights and is
checked by exact root isolation of the resulting R.  It reproduces the optimal
ISB_n the paper prints for order 4 up to 28 and order 8 up to 22 and 30
(Sec. 3.8, Table 2) and the optimum on the counts of the paper's GBS_12,8
(0.7128).  Every split of the counts into dependent and free spans the same
weights, but the LP's conditioning depends on the split.  With the short
sequences dependent, the bisection stops below Table 2 on all counts up to 36
(order 12: 0.677 against 0.7504) and 32 (order 16: 0.42 against 0.6075).  With
the longest sequence among the dependent ones and continuation, the exact ISB_n
of the returned weights is 0.75042 at order 12, 0.63534 at order 16 and 0.85587
at order 8 up to 40 (printed 0.8551).
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


def affine_weights_exact(order, steps_dep, steps_free):
    """c = c0 + G c_free with c = (c_dep, c_free), as exact rationals: c0 (a list of m) and G
    (m lists of |free|)."""
    q = order // 2
    Vd = _vandermonde(steps_dep, order)
    Vf = _vandermonde(steps_free, order)
    b = [Fraction(1)] + [Fraction(0)] * (q - 1)
    m, nf = len(steps_dep) + len(steps_free), len(steps_free)
    c0 = [Fraction(0)] * m
    c0[:q] = _solve(Vd, b)
    G = [[Fraction(0)] * nf for _ in range(m)]
    for f in range(nf):
        col = _solve(Vd, [-Vf[j][f] for j in range(q)])
        for i in range(q):
            G[i][f] = col[i]
        G[q + f][f] = Fraction(1)
    return c0, G


def affine_weights(order, steps_dep, steps_free):
    """c = c0 + G c_free with c = (c_dep, c_free): c0 and G of affine_weights_exact in FP64."""
    c0, G = affine_weights_exact(order, steps_dep, steps_free)
    return np.array([float(v) for v in c0]), np.array([[float(v) for v in row] for row in G])


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


class _DeltaRows:
    """delta(xi) = e^(-xi) R(xi) - 1 on the contour xi = i h y, affine in the free weights:
    delta = d0 + D c_free.  |R| <= 1 is |1 + delta| <= 1, and delta carries no cancellation
    against 1: for |xi| <= XS it is summed from the exact Taylor coefficients of R - e^xi, whose
    first p + 1 vanish by the order constraints (Sec. 3.2), so near the origin, where delta is
    O(xi^(p+1)), it keeps its relative accuracy; further out from the GBS recurrence."""

    XS = 6.0

    def __init__(self, order, steps, c0x, Gx):
        self.order, self.steps = order, tuple(steps)
        deg = max(steps) + 1
        coef = [gbs_poly_coeffs(n, deg) for n in steps]           # exact, m x (deg + 1)
        nf = len(Gx[0])
        E0, Q = [], []
        for j in range(order + 1, deg + 1):
            E0.append(float(sum(c0x[k] * coef[k][j] for k in range(len(steps))) - Fraction(1, factorial(j))))
            Q.append([float(sum(Gx[k][f] * coef[k][j] for k in range(len(steps)))) for f in range(nf)])
        self.j0, self.deg = order + 1, deg
        self.E0, self.Q = np.array(E0), np.array(Q)                 # (deg - p) and (deg - p) x nf
        self.tail = np.array([1.0 / factorial(j) for j in range(deg + 1, deg + 25)])
        self.c0 = np.array([float(v) for v in c0x])
        self.G = np.array([[float(v) for v in row] for row in Gx])

    def at(self, h, ys, x0):
        """(delta at c_free = x0, D) for the samples y (complex arrays)."""
        xi = 1j * h * ys
        small = np.abs(xi) <= self.XS
        d = np.empty(ys.size, complex)
        D = np.empty((ys.size, self.G.shape[1]), complex)
        if small.any():
            z = xi[small]
            pw = z[:, None] ** np.arange(self.j0, self.deg + 1)[None, :]
            tail = -(z[:, None] ** np.arange(self.deg + 1, self.deg + 25)[None, :]) @ self.tail
            em = np.exp(-z)
            d[small] = em * (pw @ (self.E0 + self.Q @ x0) + tail)
            D[small] = em[:, None] * (pw @ self.Q)
        big = ~small
        if big.any():
            z = xi[big]
            P = np.stack([gbs_poly_values(n, z) for n in self.steps], axis=1)
            em = np.exp(-z)
            d[big] = em * (P @ (self.c0 + self.G @ x0)) - 1.0
            D[big] = em[:, None] * (P @ self.G)
        return d, D


def _excess(d):
    """|1 + delta| - 1 without cancellation."""
    return (2.0 * d.real + np.abs(d) ** 2) / (np.abs(1.0 + d) + 1.0)


def _max_excess(h, rows_model, x, grid, zooms=2, pts=201):
    """Largest |R(i h y)| - 1 over y in (0, 1] for the weights x: on the grid, then around every
    local maximum of the grid on windows of pts samples spanning two grid steps, zooming twice
    (|R| oscillates in y, and a peak between grid samples can exceed the circle while every
    sample stays inside; delta keeps its relative accuracy, so the grid's local maxima are the
    oscillations', a few dozen)."""
    e = _excess(rows_model.at(h, grid, x)[0])
    best = float(e.max())
    inner = np.arange(1, e.size - 1)
    peaks = inner[(e[inner] >= e[inner - 1]) & (e[inner] >= e[inner + 1])]
    if peaks.size == 0:
        return best
    ys, width = grid[peaks], float(grid[1] - grid[0])
    for _ in range(zooms):
        win = np.clip(ys[:, None] + np.linspace(-width, width, pts)[None, :], grid[0], grid[-1])
        ee = _excess(rows_model.at(h, win.ravel(), x)[0]).reshape(win.shape)
        best = max(best, float(ee.max()))
        ys = win[np.arange(win.shape[0]), ee.argmax(axis=1)]
        width *= 2.0 / (pts - 1)
    return best


def _lp_feasible(h, rows_model, lead, order, ys, margin, x0, tol=1e-10, angles=8, rounds=60, slack=0.0):
    """Free weights with |1 + delta_j| <= 1 - mu_j on the samples and the lead term negative, by
    cutting planes around x0: the half-planes Re(e^(-i psi) delta_j) <= 1 - cos psi - mu_j, cut
    at psi = arg(1 + delta_j), each row scaled by its own sensitivity to the free weights;
    converged when every sample's excess is below tol times its sensitivity.  (x, column
    scales), or None if the LP proves that none exists or the cuts do not settle.  slack: |R| may
    exceed 1 by that much; lead None: no constraint at the origin."""
    d, B = rows_model.at(h, ys, x0)
    Dc = 1.0 / np.maximum(np.abs(B).max(axis=0), 1e-300)     # column scaling: x = x0 + Dc z
    Bs = B * Dc[None, :]
    sens = np.maximum(np.abs(Bs).max(axis=1), 1e-300)
    mu = _margin(h, ys, margin, order) - slack
    nf = Bs.shape[1]
    rows, rhs = [], []

    def cut(j, psi):
        e = np.exp(-1j * psi)
        r = (e * Bs[j]).real
        sc = 1.0 / max(np.abs(r).max(), sens[j])
        rows.append(np.concatenate([r * sc, [-sens[j] * sc]]))
        rhs.append((2.0 * np.sin(0.5 * psi) ** 2 - mu[j] - (e * d[j]).real) * sc)

    for j in range(d.size):
        for k in range(angles):
            cut(j, 2 * np.pi * k / angles)
    extra_rows, extra_rhs = [], []
    if lead is not None:
        lg, lr = lead
        eps = 1e-8 * abs(lr)
        ls = 1.0 / max(np.abs(lg * Dc).max(), 1e-300)
        extra_rows.append(np.concatenate([lg * Dc * ls, [0.0]]))
        extra_rhs.append(-(lr + lg @ x0 + eps) * ls)
    cost = np.zeros(nf + 1)
    cost[-1] = 1.0
    bounds = [(None, None)] * nf + [(-1.0, None)]
    for _ in range(rounds):
        A_ub, b_ub = np.array(rows + extra_rows), np.array(rhs + extra_rhs)
        res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs-ds")
        if res.status == 4:   # numerical trouble in the simplex: try the interior-point method
            res = linprog(cost, A_ub=A_ub, b_ub=b_ub, bounds=bounds, method="highs-ipm")
        if res.status != 0 or res.x[-1] > 0:
            return None
        z = res.x[:nf]
        dz = d + Bs @ z
        v = (_excess(dz) + mu) / sens
        if v.max() <= tol:
            return x0 + z * Dc, Dc
        for j in np.where(v > tol)[0]:
            cut(j, np.arctan2(dz[j].imag, 1.0 + dz[j].real))
    return None


def _feasible(h, rows_model, lead, order, ys, fine, margin, x0, tol=1e-10, rounds=8, slack=0.0):
    """Exchange loop around the LP: weights stable on the fine grid (half the margin), or None."""
    pts = ys
    for _ in range(rounds):
        r = _lp_feasible(h, rows_model, lead, order, pts, margin, x0, slack=slack)
        if r is None:
            return None
        x, Dc = r
        d, B = rows_model.at(h, fine, x)
        sens = np.maximum(np.abs(B * Dc[None, :]).max(axis=1), 1e-300)
        v = (_excess(d) + 0.5 * _margin(h, fine, margin, order) - slack) / sens
        bad = np.where(v > tol)[0]
        if bad.size == 0:
            return x
        pts = np.unique(np.concatenate([pts, fine[bad]]))
    return None


def longest_dependent_split(order, steps):
    """(steps_dep, steps_free) with the order/2 - 1 shortest counts and the longest one dependent,
    the rest free: the parametrisation with which the LP, with continuation, reaches Table 2
    (orders 8 to 16 on all even counts; see optimise)."""
    s = sorted(int(n) for n in steps)
    q = order // 2
    if len(s) <= q or len(set(s)) != len(s):
        raise ValueError("need more than order/2 distinct step counts")
    dep = tuple(s[:q - 1]) + (s[-1],)
    return dep, tuple(n for n in s if n not in dep)


def optimise(order, steps_dep, steps_free, n_samples=600, refine=60, margin=1e-9, rel_tol=1e-7, h_hi=None,
             slack=0.0, origin=True, continuation=False):
    """Maximise the imaginary stability boundary over the free weights (App. B): bisection over
    h in (0, N_max + 1] with the LP feasibility test above.  The dependent/free split only fixes
    the parametrisation (every split spans the same weights), but it sets the LP's conditioning:
    at orders 8 to 16 on all even counts, the longest sequence among the dependent ones with
    continuation reaches Table 2, the short sequences alone dependent stop short.  slack > 0 accepts |R| up to 1 + slack on the contour, and origin=False
    drops the constraint at the origin: the looser criterion under which a sampled FP64
    solver at its tolerance counts a polynomial as stable (strictly stable optima need the
    defaults).  continuation: after the bisection, raise h in small steps from the weights found,
    each feasibility test started from the last feasible weights and kept only if |R| - 1 stays
    within slack + 1e-12 on the fine grid and around its local maxima (_max_excess; halving the
    step on a failure down to rel_tol): at
    orders 12 and 16 the LP is so badly conditioned that a test started far from a solution can
    miss one, and from nearby it succeeds."""
    steps_dep, steps_free = tuple(steps_dep), tuple(steps_free)
    steps = steps_dep + steps_free
    c0x, Gx = affine_weights_exact(order, steps_dep, steps_free)
    c0 = np.array([float(v) for v in c0x])
    G = np.array([[float(v) for v in row] for row in Gx])
    lead = _lead_constraint(order, steps, c0, G) if origin else None
    rows_model = _DeltaRows(order, steps, c0x, Gx)
    nmax = max(steps)
    ys = np.arange(1, n_samples + 1) / n_samples
    fine = np.arange(1, refine * n_samples + 1) / (refine * n_samples)
    lo, hi = 0.0, float(h_hi if h_hi is not None else nmax + 1)
    best = np.zeros(len(steps_free))
    found = False
    while hi - lo > rel_tol * hi:
        mid = 0.5 * (lo + hi)
        x = _feasible(mid, rows_model, lead, order, ys, fine, margin, best, slack=slack)
        if x is not None:
            lo, best, found = mid, x, True
        else:
            hi = mid
    if not found:
        raise ValueError("no stable free weights found")
    if continuation:
        step = 2e-3 * lo
        while step > rel_tol * lo:
            x = _feasible(lo + step, rows_model, lead, order, ys, fine, margin, best, slack=slack)
            # the LP's tolerance is relative to each sample's sensitivity, which is large far out
            # on the contour: a step is kept only if |R| - 1 <= slack + 1e-12 on the fine grid
            if x is not None and _max_excess(lo + step, rows_model, x, fine) <= slack + 1e-12:
                lo, best = lo + step, x
            else:
                step *= 0.5
    return OptResult(steps_dep, steps_free, best, lo, lo / (nmax + 1))


def rationalize(values, max_den=1 << 20):
    """Nearby small rationals for the free weights (the paper prints such rationals, Sec. 3.8)."""
    return [Fraction(float(v)).limit_denominator(max_den) for v in values]


GBS_6_6_STEPS = ((2, 4, 6), (8, 10, 12, 14, 16, 18, 20, 22))


def gbs_6_6_free_weights():
    """The free weights of the GBS_6,6 scheme: the order-6 optimum on all even step counts up to
    22 kept 1e-4 inside the unit circle (the margin of the LP above), rounded to rationals with
    denominators below 2^16 as the paper does for its schemes (Sec. 3.8).  The margin keeps the
    rounded weights' imaginary stability boundary at the optimiser's (exact ISB_n 0.76765); with
    the default 1e-9 the optimum is the order-8 one, and its rounding loses a third of the
    boundary.  The order-7 error term stays nonzero: the scheme is order 6, not 8."""
    dep, free = GBS_6_6_STEPS
    return rationalize(optimise(6, dep, free, margin=1e-4).c_free, (1 << 16) - 1)
