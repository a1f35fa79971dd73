"""Fully determined scheme search (Sec. 3.3) and the leading error coefficient (Sec. 3.5).

Pins:
* the search's own Vandermonde solve equals the oracle's exact solve on the printed Table 1
  sets (two independent implementations);
* its floating-point ISB scan agrees with exact root isolation (oracle) on printed schemes and
  on its own winner, and the printed Table 1 ISB_n values come out of the same ranking;
* a_(p+2) < 0 for every printed scheme of order divisible by 4 (the paper's requirement for a
  positive ISB) and > 0 for the order-6 scheme, where (i theta)^(p+2) changes sign;
* the leading error comes from the first uneliminated moment: a_(p+1) / sum_k c_k n_k^(-p) and
  a_(p+2) / a_(p+1) are the same for every scheme of one order;
* a series inversion of log R(xi) done independently with sympy gives the same a_(p+1), a_(p+2);
* |a_(p+1)| decreases from the 6-core to the 8-core optimised order-8 scheme (Sec. 3.5, Fig. 3).
"""
from fractions import Fraction

import pytest

from oracle import weights as OW
from paper_1907_11771_gb300 import schemes as S
from paper_1907_11771_gb300 import search as SR
from tests.conftest import load_golden

GOLD = load_golden("paper_schemes.txt")
TABLE1 = {8: "table1_order8", 12: "table1_order12", 16: "table1_order16"}


def _exact(s):
    if s.steps_free:
        return OW.scheme_weights(s.order, list(s.steps_dep), list(s.steps_free), [Fraction(t) for t in s.c_free_text])
    steps = list(s.steps_dep)
    return steps, OW.square_weights(steps, s.order)


@pytest.mark.parametrize("order", [8, 12, 16])
def test_square_weights_match_oracle_and_isb_scan_matches_exact(order):
    g = GOLD[TABLE1[order]]
    steps = [int(t) for t in g["dep"].split()]
    c = SR.square_weights(steps, order)
    assert c == OW.square_weights(steps, order)
    isb = SR.isb_scan(steps, c, tol=1e-13)
    exact = float(OW.isb_exact(OW.stability_poly(steps, c)))
    assert isb == pytest.approx(exact, rel=1e-9)
    assert isb / (max(steps) + 1) == pytest.approx(float(g["isb_n"]), abs=5e-5)


def test_order8_search_ranks_the_printed_scheme_and_its_winner_is_exact():
    ranked = SR.search_fully_determined(8, top=10 ** 6)
    assert len(ranked) == 495                      # all 4-subsets of {2, ..., 24}
    best = ranked[0]
    exact = float(OW.isb_exact(OW.stability_poly(list(best.steps), list(best.weights))))
    assert best.isb == pytest.approx(exact, rel=1e-9)
    printed = [s for s in ranked if s.steps == (2, 16, 18, 20)][0]
    assert printed.isb_n == pytest.approx(0.5799, abs=5e-5)
    # the printed scheme is the best one whose largest step count is 20
    assert [s for s in ranked if max(s.steps) == 20][0].steps == (2, 16, 18, 20)
    assert all(s.isb > 0 for s in ranked)          # order 8: every square scheme covers the axis


def test_leading_error_signs_moment_structure_and_decay():
    rows = {}
    for s in (S.SQ8_TABLE1, S.SQ8_2468, S.GBS_8_6, S.GBS_8_8, S.SQ12_TABLE1, S.GBS_12_8, S.SQ16_TABLE1, S.GBS_6_6):
        steps, c = _exact(s)
        a1, a2 = SR.leading_error(steps, c, s.order)
        moment = sum(Fraction(ci) / Fraction(n) ** s.order for ci, n in zip(c, steps))
        rows[s.name] = (s.order, a1, a2, a1 / moment, a2 / a1)
        if s.order % 4 == 0:
            assert a2 < 0, s.name
        else:
            assert a2 > 0, s.name
    for p in (8, 12):
        same = [r for r in rows.values() if r[0] == p]
        assert len({r[3] for r in same}) == 1 and len({r[4] for r in same}) == 1, p
    assert abs(rows["GBS_8,8"][1]) < abs(rows["GBS_8,6"][1])


def test_leading_error_matches_an_independent_series_inversion():
    sp = pytest.importorskip("sympy")
    steps, c = _exact(S.SQ8_2468)
    p = 8
    xi, th = sp.symbols("xi theta")
    R = sum(sp.Rational(ci.numerator, ci.denominator) * sum(sp.Rational(v.numerator, v.denominator) * xi ** k
                                                              for k, v in enumerate(OW.gbs_stability_poly(n)))
            for ci, n in zip(c, steps))
    L = sp.series(sp.log(R), xi, 0, p + 3).removeO()          # log R = i theta
    # invert i theta = L(xi) for xi = i theta + b1 (i theta)^(p+1) + b2 (i theta)^(p+2)
    t = sp.I * th
    b1, b2 = sp.symbols("b1 b2")
    expr = sp.expand(sp.series(L.subs(xi, t + b1 * t ** (p + 1) + b2 * t ** (p + 2)), th, 0, p + 3).removeO() - t)
    sol = sp.solve([sp.expand(expr.coeff(th, p + 1)), sp.expand(expr.coeff(th, p + 2))], [b1, b2], dict=True)[0]
    a1, a2 = SR.leading_error(steps, c, p)
    assert sp.Rational(a1.numerator, a1.denominator) == sol[b1]
    assert sp.Rational(a2.numerator, a2.denominator) == sol[b2]
