"""Fully determined extrapolation schemes (Sec. 3.3) and the leading error coefficient (Sec. 3.5).

Sec. 3.3 tries every set of p/2 even step counts up to a maximum (24 in the paper) as a
square scheme, whose weights the order constraints fix uniquely (Sec. 3.2), and keeps the
set with the largest ISB_n = ISB / (N_max + 1) (Sec. 2.2, Sec. 3.6).  ``search_fully_determined``
does this with a floating-point scan of |R(iy)| on a grid refined by bisection: it ranks the
candidates; the ISB of a chosen scheme is then confirmed by exact root isolation.

Sec. 3.5 writes the boundary of the stability domain near the origin, R(xi) = e^(i theta), as
xi(theta) = i theta + a_(p+1) (i theta)^(p+1) + a_(p+2) (i theta)^(p+2) + O(theta^(p+3)).  With
R(xi) = e^xi + e_(p+1) xi^(p+1) + e_(p+2) xi^(p+2) + ..., log R(xi) = xi + e_(p+1) xi^(p+1) +
(e_(p+2) - e_(p+1)) xi^(p+2) + O(xi^(p+3)), and inverting i theta = log R(xi) to this order gives
a_(p+1) = -e_(p+1) and a_(p+2) = e_(p+1) - e_(p+2) (``leading_error``, exact rationals).
A positive ISB needs a_(p+2) < 0 for p divisible by 4 (Sec. 3.5).
"""
import itertools
from dataclasses import dataclass
from fractions import Fraction
from math import factorial

import numpy as np

from .optimize import gbs_poly_coeffs, gbs_poly_values


def square_weights(steps, order):
    """Exact rational weights of the square Vandermonde system sum_k c_k n_k^(-2j) = [j == 0],
    j = 0..p/2-1 (Sec. 3.2)."""
    q = order // 2
    if len(steps) != q:
        raise ValueError("a square scheme has exactly order/2 step counts")
    A = [[Fraction(1, n) ** (2 * j) for n in steps] + [Fraction(int(j == 0))] for j in range(q)]
    for col in range(q):
        piv = next(r for r in range(col, q) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        A[col] = [v / A[col][col] for v in A[col]]
        for r in range(q):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return [A[i][q] for i in range(q)]


def isb_scan(steps, c, y_max=None, n_grid=4000, tol=1e-9, refine=40):
    """Floating-point ISB: the first y > 0 where |R(iy)|^2 - 1 exceeds tol, located on a uniform
    grid over (0, y_max] and refined by bisection (y_max default: N_max + 1, beyond which no
    GBS sequence stays bounded)."""
    steps = list(steps)
    c = np.array([float(v) for v in c])
    y_max = float(max(steps) + 1) if y_max is None else y_max

    def excess(y):
        P = np.stack([gbs_poly_values(n, 1j * np.atleast_1d(y)) for n in steps], axis=1)
        R = P @ c
        return R.real ** 2 + R.imag ** 2 - 1.0

    ys = np.linspace(y_max / n_grid, y_max, n_grid)
    bad = np.nonzero(excess(ys) > tol)[0]
    if bad.size == 0:
        return y_max
    i = bad[0]
    if i == 0:
        return 0.0
    lo, hi = ys[i - 1], ys[i]
    for _ in range(refine):
        mid = 0.5 * (lo + hi)
        if excess(mid)[0] > tol:
            hi = mid
        else:
            lo = mid
    return lo


@dataclass(frozen=True)
class SquareScheme:
    steps: tuple
    weights: tuple     # exact rationals
    isb: float
    isb_n: float


def search_fully_determined(order, n_max=24, top=5, **scan):
    """Rank every set of order/2 even step counts <= n_max by ISB_n (Sec. 3.3); returns the
    best `top` as SquareScheme, largest ISB_n first."""
    evens = range(2, n_max + 1, 2)
    out = []
    for steps in itertools.combinations(evens, order // 2):
        c = square_weights(steps, order)
        # |R(iy)|^2 - 1 starts with -2 a_(p+2) y^(p+2) (p divisible by 4): with a_(p+2) >= 0 the
        # modulus leaves the unit circle right at the origin, ISB = 0, whatever a float scan sees
        if order % 4 == 0 and leading_error(steps, c, order)[1] >= 0:
            isb = 0.0
        else:
            isb = isb_scan(steps, c, **scan)
        out.append(SquareScheme(tuple(steps), tuple(c), isb, isb / (max(steps) + 1)))
    out.sort(key=lambda s: -s.isb_n)
    return out[:top]


def leading_error(steps, c, order):
    """(a_(p+1), a_(p+2)) of Sec. 3.5 as exact rationals, from the Taylor coefficients of R."""
    p = order
    coef = [gbs_poly_coeffs(n, p + 2) for n in steps]
    e = {k: sum(Fraction(ci) * cf[k] for ci, cf in zip(c, coef)) - Fraction(1, factorial(k)) for k in (p + 1, p + 2)}
    return -e[p + 1], e[p + 1] - e[p + 2]
