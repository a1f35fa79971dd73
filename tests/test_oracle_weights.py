"""Pins for the oracle's weights, stability polynomials and ISB (no GPU).

Each check ties the oracle to something other than itself: rationals and ISB_n
values printed in the paper (tests/golden/paper_schemes.txt), the textbook
closed form of Richardson weights, the closed form of the leap-frog
recurrence, the Taylor series of exp, and RK4's known ISB of 2 sqrt(2).
"""
import cmath
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import weights as W
from tests.conftest import load_golden

SCHEMES = load_golden("paper_schemes.txt")


def _fr_list(s):
    return [Fraction(t) for t in s.split()]


def _int_list(s):
    return [int(t) for t in s.split()]


def scheme(name):
    sc = SCHEMES[name]
    order = int(sc["order"])
    dep = _int_list(sc["dep"])
    free = _int_list(sc.get("free", ""))
    cfree = _fr_list(sc.get("cfree", ""))
    steps, c = W.scheme_weights(order, dep, free, cfree)
    return order, steps, c, float(sc["isb_n"]), int(sc["evals"])


@pytest.mark.parametrize("name", ["table1_order8", "table1_order12"])
def test_square_weights_match_printed_rationals(name):
    sc = SCHEMES[name]
    c = W.square_weights(_int_list(sc["dep"]), int(sc["order"]))
    assert c == _fr_list(sc["c"])


@pytest.mark.parametrize("steps,order", [([2, 4], 4), ([2, 4, 6, 8], 8), ([2, 16, 18, 20], 8),
                                         ([2, 8, 12, 14, 16, 20], 12), ([2, 8, 10, 12, 14, 16, 18, 22], 16)])
def test_square_weights_equal_richardson_product_formula(steps, order):
    # Lagrange basis at h^2 = 0: c_i = prod_{l != i} n_i^2 / (n_i^2 - n_l^2)
    c = W.square_weights(steps, order)
    for i, ni in enumerate(steps):
        prod = Fraction(1)
        for l, nl in enumerate(steps):
            if l != i:
                prod *= Fraction(ni * ni, ni * ni - nl * nl)
        assert c[i] == prod


def test_textbook_richardson_2468():
    assert W.square_weights([2, 4, 6, 8], 8) == [Fraction(-1, 360), Fraction(16, 45),
                                                  Fraction(-729, 280), Fraction(1024, 315)]
    assert W.square_weights([2, 4], 4) == [Fraction(-1, 3), Fraction(4, 3)]


@pytest.mark.parametrize("name", ["gbs_8_6", "gbs_8_8", "gbs_12_8"])
def test_dependent_weights_satisfy_order_constraints_exactly(name):
    order, steps, c, _, _ = scheme(name)
    assert all(r == 0 for r in W.order_residuals(steps, c, order))
    assert sum(c) == 1


@pytest.mark.parametrize("name", ["table1_order8", "table1_order12", "table1_order16",
                                  "gbs_8_6", "gbs_8_8", "gbs_12_8"])
def test_isb_n_matches_printed_value(name):
    order, steps, c, isb_n, evals = scheme(name)
    assert evals == W.evals_per_core(steps)
    isb = W.isb_exact(W.stability_poly(steps, c))
    assert round(isb / evals, 4) == pytest.approx(isb_n, abs=1.01e-4)


def test_gbs_8_8_needs_free_count_24():
    # The printed list of free step counts is one short; dropping the 11th weight instead
    # gives an ISB_n far from the printed 0.8176.
    sc = SCHEMES["gbs_8_8"]
    cf = _fr_list(sc["cfree"])[:10]
    steps, c = W.scheme_weights(8, _int_list(sc["dep"]), [4, 6, 8, 10, 12, 14, 16, 18, 20, 22], cf)
    isb_n = W.isb_exact(W.stability_poly(steps, c)) / 31
    assert abs(isb_n - 0.8176) > 0.05


def test_gbs_8_6_dependent_weights_values():
    _, steps, c, _, _ = scheme("gbs_8_6")
    assert steps[:4] == [2, 4, 6, 10]
    np.testing.assert_allclose([float(v) for v in c[:4]],
                               [-3.6874001566e-06, 7.2730950756e-05, 6.9543861448e-04, 8.3811606453e-03],
                               rtol=1e-9)


def test_rk4_isb_is_two_sqrt_two():
    golden = load_golden("paper_isb_other.txt")
    rk4 = [Fraction(1), Fraction(1), Fraction(1, 2), Fraction(1, 6), Fraction(1, 24)]
    isb = W.isb_exact(rk4)
    assert isb == pytest.approx(2 * math.sqrt(2), rel=1e-15)
    assert round(isb, 4) == float(golden["rk4_isb"])
    assert round(isb / 4, 4) == float(golden["rk4_isb_n"])


def test_isb_zero_for_forward_euler_and_order6_square():
    assert W.isb_exact([Fraction(1), Fraction(1)]) == 0.0
    # FZL07 (Sec. 2.2): square order-6 GBS schemes have no imaginary-axis coverage
    c = W.square_weights([2, 4, 6], 6)
    assert W.isb_exact(W.stability_poly([2, 4, 6], c)) == 0.0


@pytest.mark.parametrize("n", [2, 4, 8, 16, 22, 30])
def test_gbs_polynomial_matches_leapfrog_closed_form(n):
    # y_j = alpha r+^j + beta r-^j with r+- = z +- sqrt(1 + z^2), y_0 = 1, y_1 = 1 + z.
    P = [complex(float(a)) for a in W.gbs_stability_poly(n)]
    rng = np.random.default_rng(n)
    for _ in range(5):
        z = complex(rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3))
        s = cmath.sqrt(1 + z * z)
        rp, rm = z + s, z - s
        beta = (rp - (1 + z)) / (rp - rm)
        alpha = 1 - beta
        y = lambda j: alpha * rp ** j + beta * rm ** j
        closed = (y(n - 1) + 2 * y(n) + y(n + 1)) / 4
        assert W.poly_eval(P, n * z) == pytest.approx(closed, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("name", ["table1_order8", "table1_order12", "gbs_8_6", "gbs_8_8", "gbs_12_8"])
def test_stability_polynomial_has_order_p(name):
    # R(xi) - exp(xi) = O(xi^(p+1)) with a nonzero xi^(p+1) term (order exactly p).
    order, steps, c, _, _ = scheme(name)
    R = W.stability_poly(steps, c)
    for k in range(order + 1):
        assert R[k] == Fraction(1, math.factorial(k)), k
    assert R[order + 1] != Fraction(1, math.factorial(order + 1))


def test_single_sequence_even_power_error():
    # Sec. 2.1: for even N the error expansion has only even powers of h; on y' = y the
    # per-sequence polynomial minus exp therefore starts at xi^3 but the coefficient pattern in
    # h = xi/N has a_2 h^2 leading.  Check: P_N - exp(xi) = a_2 (xi/N)^2 xi + ... -> scaling 1/N^2.
    e3 = [W.gbs_stability_poly(n)[3] - Fraction(1, 6) for n in (2, 4, 8)]
    assert e3[0] / e3[1] == 4 and e3[1] / e3[2] == 4
