#!/usr/bin/env python3
"""Writes univariate_exact.txt: the exact univariate B-spline mass and stiffness
matrices M[i][j] = int B_i B_j, K[i][j] = int B_i' B_j' (Section 2.1, the
matrices K_hat, M_hat of Section 5.2) on [0, 1] with open uniform knots, as
exact rationals.

The basis functions are built by the Cox-de Boor recursion on exact
polynomials (Fraction coefficients, one polynomial per knot span) and
integrated exactly; no floating point and no quadrature are involved, so the
fixture is independent of the oracle's Gauss-rule assembly it pins.

    python tests/golden/make_univariate.py
"""
from fractions import Fraction as F
import os


def padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def pmul(a, b):
    out = [F(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def pder(a):
    return [i * a[i] for i in range(1, len(a))] or [F(0)]


def pint(a, lo, hi):
    return sum(c * (hi ** (i + 1) - lo ** (i + 1)) / (i + 1) for i, c in enumerate(a))


def basis(knots, p):
    """basis[i][s]: polynomial of B_{i,p} on span s = [knots[s], knots[s+1])."""
    ns = len(knots) - 1
    B = [[([F(1)] if knots[i] <= knots[s] < knots[i + 1] else [F(0)]) for s in range(ns)]
         for i in range(ns)]
    for q in range(1, p + 1):
        nb = len(knots) - q - 1
        new = []
        for i in range(nb):
            row = []
            for s in range(ns):
                acc = [F(0)]
                d1 = knots[i + q] - knots[i]
                if d1 != 0:   # (x - t_i) / d1 * B_{i,q-1}
                    acc = padd(acc, pmul([-knots[i] / d1, F(1) / d1], B[i][s]))
                d2 = knots[i + q + 1] - knots[i + 1]
                if d2 != 0:   # (t_{i+q+1} - x) / d2 * B_{i+1,q-1}
                    acc = padd(acc, pmul([knots[i + q + 1] / d2, F(-1) / d2], B[i + 1][s]))
                row.append(acc)
            new.append(row)
        B = new
    return B


def matrices(p, nel):
    knots = [F(0)] * p + [F(j, nel) for j in range(nel + 1)] + [F(1)] * p
    B = basis(knots, p)
    n = nel + p
    M = [[F(0)] * n for _ in range(n)]
    K = [[F(0)] * n for _ in range(n)]
    for s in range(len(knots) - 1):
        lo, hi = knots[s], knots[s + 1]
        if lo == hi:
            continue
        for i in range(n):
            for j in range(n):
                M[i][j] += pint(pmul(B[i][s], B[j][s]), lo, hi)
                K[i][j] += pint(pmul(pder(B[i][s]), pder(B[j][s])), lo, hi)
    return M, K


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "univariate_exact.txt")
    with open(path, "w") as f:
        f.write("# Exact univariate B-spline mass M and stiffness K on [0,1], open uniform knots.\n")
        f.write("# Written by tests/golden/make_univariate.py (exact rational Cox-de Boor\n")
        f.write("# polynomials, exact integration).  Definition: Section 2.1 (B-splines) and the\n")
        f.write("# univariate matrices K_hat, M_hat of Section 5.2.  Format: 'p nel' then n rows\n")
        f.write("# of M, then n rows of K, entries as num/den.\n")
        for p, nel in ((2, 2), (2, 3), (3, 3), (4, 5)):
            M, K = matrices(p, nel)
            f.write(f"case {p} {nel}\n")
            for A in (M, K):
                for row in A:
                    f.write(" ".join(f"{x.numerator}/{x.denominator}" for x in row) + "\n")


if __name__ == "__main__":
    main()
