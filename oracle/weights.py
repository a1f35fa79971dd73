"""Exact extrapolation weights, stability polynomials and ISB (oracle side).

Everything here works in exact rational arithmetic (``fractions.Fraction``)
and is rounded to FP64 only at the very end, as the paper asks for the
dependent weights (Sec. 3.7: they are best computed symbolically and only then
converted to floating point).

Paper passages followed:

* Sec. 3.2, eq. "vander": for step counts n_1..n_m and h_i = H/n_i, the order
  constraints for a GBS extrapolation of order p are the p/2 equations
  sum_i c_i h_i^(2j) = [j == 0], j = 0..p/2-1.  The weights do not depend on
  H (row j scales by H^(2j) and its right-hand side is 0 for j > 0), so
  h_i = 1/n_i is used throughout.
* Sec. 3.7, eqs. "order_constraints" and "cdep_computation":
  c_dep = V_dep^-1 (b - V_free c_free).
* Sec. 2.1 eq. "GBS" applied to Dahlquist's test equation y' = lambda y
  (Appendix A, eq. "SD_ODE"): the stability polynomial P_n(xi), xi = H lambda,
  of one sequence with n steps; Appendix B: R(xi) = sum_i c_i P_i(xi).
* Sec. 2.2: ISB is the largest y with [-iy, iy] inside {|R| <= 1}; 0 if none.
  ISB_n divides by the function evaluations per core (Sec. 3.6: with pair
  folding and the shared first evaluation, N_max + 1).
"""
from fractions import Fraction

import sympy


# ---------------------------------------------------------------------------
# Order constraints (Sec. 3.2 eq. "vander"; Sec. 3.7)
# ---------------------------------------------------------------------------

def vandermonde(steps, order):
    """The (order/2) x m matrix V of eq. "vander" with h_i = 1/n_i, as Fractions."""
    if order % 2:
        raise ValueError("GBS order must be even")
    rows = order // 2
    return [[Fraction(1, n) ** (2 * j) for n in steps] for j in range(rows)]


def rhs_b(order):
    """Right-hand side b = (1, 0, ..., 0) of eq. "vander"."""
    return [Fraction(1)] + [Fraction(0)] * (order // 2 - 1)


def solve_exact(A, b):
    """Solve the square rational system A x = b by plain Gauss-Jordan elimination
    (Sec. 3.2 eq. "vander", Sec. 3.7 eq. "cdep_computation")."""
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


def square_weights(steps, order):
    """Richardson weights of the square system (m = p/2), Sec. 3.2."""
    if len(steps) != order // 2:
        raise ValueError("square system needs exactly order/2 step counts")
    return solve_exact(vandermonde(steps, order), rhs_b(order))


def dependent_weights(order, steps_dep, steps_free, c_free):
    """c_dep = V_dep^-1 (b - V_free c_free), Sec. 3.7 eq. "cdep_computation"."""
    Vd = vandermonde(steps_dep, order)
    Vf = vandermonde(steps_free, order) if steps_free else [[] for _ in Vd]
    b = rhs_b(order)
    r = [b[j] - sum((Vf[j][i] * Fraction(c_free[i]) for i in range(len(steps_free))), Fraction(0))
         for j in range(len(b))]
    return solve_exact(Vd, r)


def scheme_weights(order, steps_dep, steps_free=(), c_free=()):
    """Full step-count list and exact weight list (dependent first, then free); Sec. 3.7."""
    c_dep = dependent_weights(order, list(steps_dep), list(steps_free), list(c_free))
    return list(steps_dep) + list(steps_free), c_dep + [Fraction(c) for c in c_free]


def order_residuals(steps, c, order):
    """sum_i c_i h_i^(2j) - b_j for j = 0..p/2-1, exactly: the order constraints of Sec. 3.7."""
    V = vandermonde(steps, order)
    b = rhs_b(order)
    return [sum((V[j][i] * Fraction(c[i]) for i in range(len(steps))), Fraction(0)) - b[j]
            for j in range(len(b))]


def to_fp64(c):
    """Sec. 3.8 gives rational weights; the library runs on their FP64 values.
    Round exact weights to nearest FP64 (Python's Fraction -> float rounds correctly)."""
    return [float(Fraction(v)) for v in c]


# ---------------------------------------------------------------------------
# Stability polynomials (Sec. 2.1 eq. "GBS" on y' = lambda y; Appendix B)
# Polynomials are lists of Fraction coefficients, lowest degree first.
# ---------------------------------------------------------------------------

def _padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def _pscale(a, s):
    return [s * v for v in a]


def _pshift(a):  # multiply by xi
    return [Fraction(0)] + list(a)


def gbs_stability_poly(n):
    """Stability polynomial (App. A.1) of one sequence of Sec. 2.1 eq. "GBS".
    P_n(xi): one GBS sequence with n steps of h = H/n on y' = lambda y, xi = H lambda.

    With z = h lambda = xi/n: y_0 = 1, y_1 = y_0 + z y_0 (FE), y_(j+1) = y_(j-1) + 2 z y_j
    for j = 1..n (LF), P = (y_(n-1) + 2 y_n + y_(n+1)) / 4 (averaging).
    """
    zfac = Fraction(1, n)
    ys = [[Fraction(1)]]
    ys.append(_padd(ys[0], _pscale(_pshift(ys[0]), zfac)))
    for j in range(1, n + 1):
        ys.append(_padd(ys[j - 1], _pscale(_pshift(ys[j]), 2 * zfac)))
    return _pscale(_padd(_padd(ys[n - 1], _pscale(ys[n], 2)), ys[n + 1]), Fraction(1, 4))


def stability_poly(steps, c):
    """R(xi) = sum_i c_i P_i(xi) (Appendix B)."""
    R = [Fraction(0)]
    for n, ci in zip(steps, c):
        R = _padd(R, _pscale(gbs_stability_poly(n), Fraction(ci)))
    while len(R) > 1 and R[-1] == 0:
        R.pop()
    return R


def poly_eval(coeffs, x):
    """Evaluate a coefficient list at x (Horner); x may be complex or Fraction (helper)."""
    acc = 0
    for a in reversed(coeffs):
        acc = acc * x + a
    return acc


# ---------------------------------------------------------------------------
# ISB by exact real-root isolation (Sec. 2.2)
# ---------------------------------------------------------------------------

def _abs2_minus_one(R):
    """Coefficients in s = y^2 of |R(iy)|^2 - 1 (an even polynomial in y); the ISB of
    Sec. 2.2 is where it first turns positive for y > 0."""
    # R(iy) = sum a_k i^k y^k ; Re = sum_{k even} a_k (-1)^(k/2) y^k ; Im = sum_{k odd} a_k (-1)^((k-1)/2) y^k
    re = [Fraction(0)] * len(R)
    im = [Fraction(0)] * len(R)
    for k, a in enumerate(R):
        if k % 2 == 0:
            re[k] = a * (-1) ** (k // 2)
        else:
            im[k] = a * (-1) ** ((k - 1) // 2)

    def pmul(a, b):
        out = [Fraction(0)] * (len(a) + len(b) - 1)
        for i, x in enumerate(a):
            if x:
                for j, y in enumerate(b):
                    out[i + j] += x * y
        return out

    q = _padd(pmul(re, re), pmul(im, im))
    q[0] -= 1
    # only even powers of y survive; express in s = y^2
    return [q[k] for k in range(0, len(q), 2)]


def isb_exact(R, eps=None, tol=0):
    """ISB of the stability polynomial R: inf{ y > 0 : |R(iy)|^2 > 1 + tol }, or 0.

    tol = 0 is the definition of Sec. 2.2.  A small positive tol (a Fraction or a float
    taken exactly) reports where |R| leaves the unit circle by more than rounding, which
    is the meaningful boundary for weights that were optimised in floating point.

    Exact: |R(iy)|^2 - 1 is a polynomial q(s) in s = y^2 with rational
    coefficients.  Its factor s^k (q(0) = 0 because R(0) = 1) is divided out, the
    remaining positive real roots are isolated by sympy into disjoint rational
    intervals, and the sign of q is evaluated exactly at a rational point between
    consecutive roots.  ISB^2 is the root at which q first turns positive.  The
    returned float is the midpoint of that root's isolating interval, refined to a
    relative width below ``eps`` (default 1e-18).
    """
    qs = _abs2_minus_one(R)
    qs[0] -= Fraction(tol)
    k = 0
    while k < len(qs) and qs[k] == 0:
        k += 1
    if k == len(qs):
        return float("inf")          # |R(iy)| == 1 identically
    qs = qs[k:]
    s = sympy.symbols("s")
    poly = sympy.Poly([sympy.Rational(v.numerator, v.denominator) for v in reversed(qs)], s)
    ivs = sorted((a, b) for (a, b), _m in poly.intervals(eps=sympy.Rational(1, 10 ** 12)) if b > 0)
    prev = None                      # isolating interval of the previous positive root
    for iv in ivs + [None]:
        a, b = iv if iv is not None else (None, None)
        lo = prev[1] if prev else sympy.Rational(0)
        probe = (lo + a) / 2 if iv is not None else lo + 1
        if poly.eval(probe) > 0:     # |R(iy)| > 1 right after the previous root
            break
        if iv is None:
            return float("inf")
        prev = iv
    if prev is None:
        return 0.0
    tol = sympy.Rational(1, 10 ** 18) if eps is None else sympy.Rational(str(eps))
    a, b = poly.refine_root(prev[0], prev[1], eps=tol * prev[1])
    return float(sympy.sqrt((a + b) / 2).evalf(30))


def evals_per_core(steps):
    """N_max + 1: function evaluations per core with pair folding and a shared first RHS (Sec. 3.6)."""
    return max(steps) + 1
