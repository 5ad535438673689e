"""B-splines, Gauss quadrature and the univariate matrices (Section 2.1; the
univariate stiffness/mass matrices of Section 5.2).  Oracle code: test
infrastructure only."""
from __future__ import annotations

import numpy as np


def open_knots(nel: int, p: int) -> np.ndarray:
    """Open uniform knot vector: p+1 repeated end knots, single interior knots
    (Section 2.1).  Length nel + 2p + 1, giving m = nel + p basis functions."""
    inner = [j / nel for j in range(1, nel)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1), dtype=np.float64)


def _ratio(num, den):
    """num/den with the 0/0 = 0 convention of the Cox-de Boor recursion."""
    return np.where(den == 0.0, 0.0, num / np.where(den == 0.0, 1.0, den))


def basis(knots: np.ndarray, p: int, x: np.ndarray, deriv: int = 0) -> np.ndarray:
    """Values (deriv=0) or first derivatives (deriv=1) of all m B-splines of
    degree p at the points x, by the Cox-de Boor recursion of Section 2.1.
    Returns [len(x), m].  At x = 1 the last non-empty span is taken closed so
    that b_m(1) = 1 (endpoint interpolation)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nk = len(knots)
    m = nk - p - 1
    # degree 0
    B = np.zeros((len(x), nk - 1))
    for i in range(nk - 1):
        B[:, i] = (knots[i] <= x) & (x < knots[i + 1])
    last = max(i for i in range(nk - 1) if knots[i] < knots[i + 1])
    B[x == knots[-1], last] = 1.0
    for q in range(1, p + 1):
        Bn = np.zeros((len(x), nk - 1 - q))
        for i in range(nk - 1 - q):
            left = _ratio(x - knots[i], knots[i + q] - knots[i]) * B[:, i]
            right = _ratio(knots[i + q + 1] - x, knots[i + q + 1] - knots[i + 1]) * B[:, i + 1]
            Bn[:, i] = left + right
        if q == p and deriv == 1:
            # derivative from the degree p-1 values (standard differentiation
            # of the recursion): b'_{i,p} = p/(xi_{i+p}-xi_i) b_{i,p-1}
            #                              - p/(xi_{i+p+1}-xi_{i+1}) b_{i+1,p-1}
            D = np.zeros((len(x), m))
            for i in range(m):
                a = _ratio(np.float64(p), knots[i + p] - knots[i]) * B[:, i]
                b = _ratio(np.float64(p), knots[i + p + 1] - knots[i + 1]) * B[:, i + 1]
                D[:, i] = a - b
            return D
        B = Bn
    if deriv == 1 and p == 0:
        return np.zeros((len(x), m))
    return B[:, :m]


def greville(knots: np.ndarray, p: int) -> np.ndarray:
    m = len(knots) - p - 1
    return np.array([knots[i + 1:i + p + 1].mean() if p > 0 else knots[i] for i in range(m)])


def gauss(nq: int):
    """Gauss-Legendre nodes/weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def quadrature(knots: np.ndarray, p: int, nq: int | None = None):
    """Element-wise Gauss rule with nq (default p+1) points per non-empty span.
    Returns (points, weights, element index of each point)."""
    nq = p + 1 if nq is None else nq
    g, w = gauss(nq)
    pts, wts, el = [], [], []
    e = 0
    for i in range(len(knots) - 1):
        a, b = knots[i], knots[i + 1]
        if b > a:
            pts.append(a + (b - a) * g)
            wts.append((b - a) * w)
            el.append(np.full(nq, e))
            e += 1
    return np.concatenate(pts), np.concatenate(wts), np.concatenate(el)


def univariate_matrices(nel: int, p: int):
    """1D parametric stiffness K and mass M over all m = nel+p basis functions,
    including the end (interface) functions (Section 5.2):
        K_ij = int_0^1 b_i' b_j',   M_ij = int_0^1 b_i b_j."""
    kn = open_knots(nel, p)
    x, w, _ = quadrature(kn, p)
    B0 = basis(kn, p, x)
    B1 = basis(kn, p, x, deriv=1)
    K = B1.T @ (w[:, None] * B1)
    M = B0.T @ (w[:, None] * B0)
    return K, M
