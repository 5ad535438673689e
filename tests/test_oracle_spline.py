"""Pins for the oracle's B-splines and univariate matrices (Section 2.1,
Section 5.2): partition of unity, linear and quadratic precision (Marsden's
identity), endpoint interpolation, derivative against finite differences,
the closed-form p = 1 matrices and the identities K 1 = 0, 1^T M 1 = 1,
g^T K g = 1 (Greville points), (M 1)_i = (xi_{i+p+1} - xi_i)/(p+1)."""
import itertools

import numpy as np
import pytest

from oracle import spline


@pytest.mark.parametrize("p,nel", [(1, 5), (2, 4), (3, 7), (4, 6), (5, 9)])
def test_partition_of_unity_and_endpoints(p, nel):
    kn = spline.open_knots(nel, p)
    x = np.concatenate([[0.0, 1.0], np.random.default_rng(1).uniform(0, 1, 200), kn])
    B = spline.basis(kn, p, x)
    assert B.shape[1] == nel + p
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-14)
    assert (B >= -1e-15).all()
    assert B[0, 0] == 1.0 and B[1, -1] == 1.0


@pytest.mark.parametrize("p,nel", [(1, 5), (2, 4), (3, 7), (4, 6), (5, 9)])
def test_marsden_precision(p, nel):
    """sum_i g_i b_i(x) = x and, for p >= 2, sum_i s_i b_i(x) = x^2 with
    s_i the symmetric mean of the products of pairs of interior knots."""
    kn = spline.open_knots(nel, p)
    x = np.random.default_rng(2).uniform(0, 1, 300)
    B = spline.basis(kn, p, x)
    g = spline.greville(kn, p)
    np.testing.assert_allclose(B @ g, x, atol=1e-13)
    if p >= 2:
        s = []
        for i in range(nel + p):
            ks = kn[i + 1:i + p + 1]
            pairs = [a * b for a, b in itertools.combinations(ks, 2)]
            s.append(np.mean(pairs))
        np.testing.assert_allclose(B @ np.array(s), x * x, atol=1e-13)


@pytest.mark.parametrize("p,nel", [(1, 4), (2, 5), (3, 6), (5, 7)])
def test_derivative_matches_finite_differences(p, nel):
    kn = spline.open_knots(nel, p)
    # stay away from knots where derivatives of low degree jump
    x = (np.arange(nel) + 0.37) / nel
    h = 1e-6
    D = spline.basis(kn, p, x, deriv=1)
    Dfd = (spline.basis(kn, p, x + h) - spline.basis(kn, p, x - h)) / (2 * h)
    np.testing.assert_allclose(D, Dfd, atol=1e-6 * nel * p)


def test_linear_closed_forms():
    nel = 6
    h = 1.0 / nel
    K, M = spline.univariate_matrices(nel, 1)
    n = nel + 1
    Mx = np.diag(np.full(n, 4.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    Mx[0, 0] = Mx[-1, -1] = 2.0
    Kx = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    Kx[0, 0] = Kx[-1, -1] = 1.0
    np.testing.assert_allclose(M, h / 6 * Mx, atol=1e-15)
    np.testing.assert_allclose(K, Kx / h, atol=1e-12)


@pytest.mark.parametrize("p,nel", [(2, 8), (3, 16), (4, 5), (5, 12)])
def test_univariate_identities(p, nel):
    K, M = spline.univariate_matrices(nel, p)
    kn = spline.open_knots(nel, p)
    n = nel + p
    one = np.ones(n)
    np.testing.assert_allclose(K @ one, 0.0, atol=1e-10 * nel)
    assert abs(one @ M @ one - 1.0) < 1e-14
    g = spline.greville(kn, p)
    assert abs(g @ K @ g - 1.0) < 1e-12
    np.testing.assert_allclose(M @ one, [(kn[i + p + 1] - kn[i]) / (p + 1) for i in range(n)],
                               atol=1e-15)
    np.testing.assert_allclose(K, K.T, atol=1e-12)
    np.testing.assert_allclose(M, M.T, atol=1e-15)
