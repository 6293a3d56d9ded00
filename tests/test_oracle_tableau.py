"""Pins of the oracle's Dormand-Prince tableau and dense output (App. A:
dopri5; Sec. 3: FSAL/SSAL and Horner dense output) against exact rational
arithmetic: order conditions, FSAL/SSAL structure, the continuous extension's
end and order conditions."""
from fractions import Fraction as F

import numpy as np
import pytest
import sympy as sp

import oracle
import rk_exact as rk


def test_tree_enumeration_counts():
    # numbers of rooted trees of order 1..5 (OEIS A000081)
    assert [len(rk.trees(k)) for k in range(1, 6)] == [1, 1, 2, 4, 9]


def test_row_sums_and_fsal():
    c, A, b, bh = rk.tableau()
    for i in range(7):
        assert sum(A[i]) == c[i]
    # SSAL/FSAL: the last stage row equals the 5th-order weights, c7 = 1
    assert A[6] == b and c[6] == 1 and b[6] == 0


def test_order_conditions_b_order5_bhat_order4():
    c, A, b, bh = rk.tableau()
    n5 = 0
    for order in range(1, 6):
        for t in rk.trees(order):
            ph = rk.phi(t, A)
            target = F(1, rk.gamma(t))
            assert sum(b[i] * ph[i] for i in range(7)) == target, (order, t)
            n5 += 1
            if order <= 4:
                assert sum(bh[i] * ph[i] for i in range(7)) == target, (order, t)
    assert n5 == 17
    # the embedded weights are genuinely 4th order (some 5th-order tree fails)
    fails = [t for t in rk.trees(5)
             if sum(bh[i] * rk.phi(t, A)[i] for i in range(7)) != F(1, rk.gamma(t))]
    assert fails


def test_oracle_doubles_are_the_exact_rationals():
    c, A, b, bh = rk.tableau()
    oc, oa, ob, obh, oq = oracle.tableau_doubles()
    for i in range(7):
        assert oc[i] == float(c[i])
        assert ob[i] == float(b[i])
        assert obh[i] == float(bh[i])
        for j in range(7):
            assert oa[i, j] == float(A[i][j])


def test_dense_output_exact_conditions():
    c, A, b, bh = rk.tableau()
    th, polys = rk.dense_polys()
    for i in range(7):
        p = polys[i].as_expr()
        assert p.subs(th, 0) == 0
        assert p.subs(th, 1) == sp.Rational(b[i].numerator, b[i].denominator)
        dp = sp.diff(p, th)
        assert dp.subs(th, 0) == (1 if i == 0 else 0)  # y'(t_n) = k1
        assert dp.subs(th, 1) == (1 if i == 6 else 0)  # y'(t_n+h) = k7 (C1 joint)
    # continuous order conditions up to order 4
    for order in range(1, 5):
        for t in rk.trees(order):
            ph = rk.phi(t, A)
            lhs = sum(polys[i].as_expr() * sp.Rational(ph[i].numerator, ph[i].denominator)
                      for i in range(7))
            assert sp.expand(lhs - th**order / rk.gamma(t)) == 0, (order, t)


def test_oracle_dense_coefficients_match_hnw_form():
    """The oracle's Horner coefficients are the expansion of the HNW form."""
    _, _, _, _, oq = oracle.tableau_doubles()
    th, polys = rk.dense_polys()
    for i in range(7):
        coeffs = polys[i].all_coeffs()[::-1]  # theta^0 .. theta^4
        coeffs = coeffs + [0] * (5 - len(coeffs))
        assert coeffs[0] == 0
        for k in range(4):
            exact = sp.Rational(coeffs[k + 1])
            assert oq[i, k] == float(exact), (i, k)


@pytest.mark.parametrize("theta", [0.0, 0.125, 0.5, 0.8125, 1.0])
def test_oracle_dense_weights_values(theta):
    th, polys = rk.dense_polys()
    w = oracle.dense_weights(theta)
    for i in range(7):
        assert abs(w[i] - float(polys[i].as_expr().subs(th, sp.Rational(theta)))) < 1e-15
