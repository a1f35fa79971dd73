"""The App. B stability optimiser and the optimised order-6 scheme it produced (no GPU).

The paper prints no order-6 scheme (square order-6 GBS schemes have ISB 0, Sec. 2.2), so
the optimised one is pinned by exact arithmetic only: it satisfies the order-6 constraints
exactly, its stability polynomial has order exactly 6, and its ISB, found by exact root
isolation, is the value recorded with it.  The optimiser itself is checked on a small case
against the exact ISB of the weights it returns.  (Its optimality is not pinned to the
paper's Table 2: that needs the continuous constraint, see the module docstring.)
"""
import math
from fractions import Fraction

import pytest

from oracle import weights as W
from paper_1907_11771_gb300 import optimize as O
from paper_1907_11771_gb300 import schemes as S


def _exact(sc):
    steps, c = W.scheme_weights(sc.order, list(sc.steps_dep), list(sc.steps_free),
                                [Fraction(t) for t in sc.c_free_text])
    return steps, c


def test_order6_scheme_constraints_order_and_isb():
    sc = S.GBS_6_6
    steps, c = _exact(sc)
    assert all(r == 0 for r in W.order_residuals(steps, c, 6))
    R = W.stability_poly(steps, c)
    for k in range(7):
        assert R[k] == Fraction(1, math.factorial(k))
    assert R[7] != Fraction(1, math.factorial(7))
    isb = W.isb_exact(R)
    assert isb == pytest.approx(15.00302, abs=2e-5)
    assert round(isb / sc.evals_per_core, 5) == 0.65231
    # versus the square order-6 scheme on the dependent counts: no imaginary-axis coverage
    sq = W.square_weights([2, 4, 6], 6)
    assert W.isb_exact(W.stability_poly([2, 4, 6], sq)) == 0.0


def test_optimiser_small_case_agrees_with_exact_isb():
    dep, free = (2, 4, 6), (8, 10, 12)
    r = O.optimise(6, dep, free, h_lo=2.0, n_samples=300, iters=20)
    steps, c = W.scheme_weights(6, list(dep), list(free), [Fraction(v) for v in r.c_free])
    exact = W.isb_exact(W.stability_poly(steps, c))
    assert exact > 0
    assert exact == pytest.approx(r.isb, rel=2e-2)
    # constraints hold exactly whatever the free weights are
    assert all(v == 0 for v in W.order_residuals(steps, c, 6))
