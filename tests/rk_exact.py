"""Exact-rational Runge-Kutta helpers for the tests: the golden tableau
reader, rooted trees with their elementary weights, and the stability /
error polynomials of the linear test equation."""
from __future__ import annotations

import os
from fractions import Fraction as F

import sympy as sp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def tableau():
    c = [F(0)] * 7
    A = [[F(0)] * 7 for _ in range(7)]
    b = [F(0)] * 7
    bh = [F(0)] * 7
    for r in _read("dopri5_tableau.txt"):
        if r[0] == "c":
            c[int(r[1]) - 1] = F(r[2])
        elif r[0] == "a":
            A[int(r[1]) - 1][int(r[2]) - 1] = F(r[3])
        elif r[0] == "b":
            b[int(r[1]) - 1] = F(r[2])
        elif r[0] == "bhat":
            bh[int(r[1]) - 1] = F(r[2])
    return c, A, b, bh


def dense_d():
    d = [F(0)] * 7
    for r in _read("dopri5_dense_hnw.txt"):
        d[int(r[1]) - 1] = F(r[2])
    return d


def dense_polys():
    """b_i(theta) as sympy polynomials, built from the HNW form."""
    _, _, b, _ = tableau()
    d = dense_d()
    th = sp.Symbol("theta")
    out = []
    for i in range(7):
        d1 = 1 if i == 0 else 0
        d7 = 1 if i == 6 else 0
        bi = sp.Rational(b[i].numerator, b[i].denominator)
        di = sp.Rational(d[i].numerator, d[i].denominator)
        p = (th * bi + th * (1 - th) * (d1 - bi) + th**2 * (1 - th) * (2 * bi - d1 - d7)
             + th**2 * (1 - th) ** 2 * di)
        out.append(sp.Poly(sp.expand(p), th))
    return th, out


# ---- rooted trees (Butcher) ----
def trees(order):
    """All rooted trees with exactly ``order`` nodes, as sorted tuples of
    child subtrees (the single node is ())."""
    if order == 1:
        return [()]
    res = set()

    def parts(n, maxpart):
        # multisets of subtree orders summing to n
        if n == 0:
            yield []
            return
        for k in range(min(n, maxpart), 0, -1):
            for rest in parts(n - k, k):
                yield [k] + rest

    for p in parts(order - 1, order - 1):
        def combos(idx):
            if idx == len(p):
                yield []
                return
            for t in trees(p[idx]):
                for rest in combos(idx + 1):
                    yield [t] + rest
        for cs in combos(0):
            res.add(tuple(sorted(cs)))
    return sorted(res)


def tree_order(t):
    return 1 + sum(tree_order(s) for s in t)


def gamma(t):
    g = tree_order(t)
    for s in t:
        g *= gamma(s)
    return g


def phi(t, A):
    """Elementary weight vector Phi(t) (so that b^T Phi(t) = 1/gamma(t))."""
    n = len(A)
    v = [F(1)] * n
    for s in t:
        ps = phi(s, A)
        w = [sum(A[i][j] * ps[j] for j in range(n)) for i in range(n)]
        v = [v[i] * w[i] for i in range(n)]
    return v


def linear_step_polys():
    """For y' = lambda y and z = h*lambda: (R(z), E(z)) with y1 = R y0 and
    the embedded error estimate e = E y0 (exact rationals, sympy)."""
    _, A, b, bh = tableau()
    z = sp.Symbol("z")
    n = 7
    # k/(lambda y0) = (I - zA)^{-1} 1 = sum_m z^m A^m 1 (A is nilpotent)
    stage = [sp.Integer(1)] * n
    term = [sp.Integer(1)] * n
    for m in range(1, n + 1):
        term = [sum(sp.Rational(A[i][j].numerator, A[i][j].denominator) * term[j]
                    for j in range(n)) for i in range(n)]
        stage = [stage[i] + z**m * term[i] for i in range(n)]
    R = 1 + z * sum(sp.Rational(b[i].numerator, b[i].denominator) * stage[i] for i in range(n))
    E = z * sum(sp.Rational((b[i] - bh[i]).numerator, (b[i] - bh[i]).denominator) * stage[i]
                for i in range(n))
    return z, sp.expand(R), sp.expand(E)


# ---- tsit5 (decimals as published, read as exact rationals) ----
def tsit5_tableau():
    """(c, A, b, e) of the Tsitouras 5(4) pair as exact rationals of the
    published decimals; b is the last stage row (FSAL), e = b - bhat."""
    c = [F(0)] * 7
    A = [[F(0)] * 7 for _ in range(7)]
    e = [F(0)] * 7
    for r in _read("tsit5_tableau.txt"):
        if r[0] == "c":
            c[int(r[1]) - 1] = F(r[2])
        elif r[0] == "a":
            A[int(r[1]) - 1][int(r[2]) - 1] = F(r[3])
        elif r[0] == "e":
            e[int(r[1]) - 1] = F(r[2])
    return c, A, list(A[6]), e


def tsit5_dense_polys():
    """b_i(theta) of tsit5's continuous extension as sympy polynomials with
    the published decimals read as exact rationals."""
    th = sp.Symbol("theta")
    out = [None] * 7
    for r in _read("tsit5_tableau.txt"):
        if r[0] == "bt":
            expr = sp.sympify(r[2], locals={"theta": th}, rational=True)
            out[int(r[1]) - 1] = sp.Poly(sp.expand(expr), th)
    return th, out
