"""Pins of the oracle's nested non-conforming interfaces (Section 2, Section 6
non-conforming test) against facts that do not come from the oracle itself:

- the refinement matrix reproduces every coarse B-spline from the fine ones
  at arbitrary points (the defining property of a nested space);
- a polynomial displacement of degree 2 per variable that vanishes on the
  boundary lies in every patch's space for p >= 2, so its coefficient vector
  (Greville collocation, patch by patch) must satisfy B c = 0, and the
  Galerkin solution for its exact body force (derivatives written out by
  hand below) must reproduce it: quadrature with p + 1 points is exact for
  these integrands on identity-mapped patches.
"""
import numpy as np
import pytest

import afi_workloads as W
from oracle import nested, spline
from oracle.ieti import AFIETI


@pytest.mark.parametrize("nel_c,nel_f,p", [(1, 2, 2), (2, 4, 2), (2, 6, 3), (3, 6, 1), (2, 8, 4), (4, 4, 2)])
def test_refinement_reproduces_coarse_basis(nel_c, nel_f, p):
    E = nested.refinement_matrix(nel_c, nel_f, p)
    x = np.random.default_rng(nel_c * 10 + nel_f + p).uniform(0.0, 1.0, 200)
    x = np.concatenate([x, [0.0, 1.0, 0.5]])
    Bc = spline.basis(spline.open_knots(nel_c, p), p, x)
    Bf = spline.basis(spline.open_knots(nel_f, p), p, x)
    np.testing.assert_allclose(Bf @ E, Bc, atol=1e-13)
    if nel_c == nel_f:
        np.testing.assert_allclose(E, np.eye(nel_c + p), atol=1e-13)


def test_refinement_rejects_non_nested():
    with pytest.raises(ValueError):
        nested.refinement_matrix(3, 4, 2)


# ------------------------------------------------------------------ polynomial
def _q(t, L):
    return t * (L - t)


def _dq(t, L):
    return L - 2.0 * t


def u_exact(X, amp, L):
    """u_i = amp_i prod_l x_l (L_l - x_l) at the points X [N, dim]."""
    P = np.prod([_q(X[:, l], L[l]) for l in range(X.shape[1])], axis=0)
    return amp[None, :] * P[:, None]


def f_exact(X, amp, L, lam, mu):
    """f = -div sigma(u) for u above:
    f_i = -(lam + mu) sum_k amp_k d_i d_k P - mu amp_i Lap P,
    with d_i d_k P = q_i' q_k' prod_{others} q (i != k) and
    d_i d_i P = -2 prod_{others} q."""
    d = X.shape[1]
    q = [_q(X[:, l], L[l]) for l in range(d)]
    dq = [_dq(X[:, l], L[l]) for l in range(d)]

    def others(excl):
        out = np.ones(X.shape[0])
        for l in range(d):
            if l not in excl:
                out = out * q[l]
        return out
    H = [[(-2.0 * others({i}) if i == k else dq[i] * dq[k] * others({i, k})) for k in range(d)]
         for i in range(d)]
    lap = sum(H[l][l] for l in range(d))
    f = np.zeros((X.shape[0], d))
    for i in range(d):
        f[:, i] = -(lam + mu) * sum(amp[k] * H[i][k] for k in range(d)) - mu * amp[i] * lap
    return f


def collocate(prob, k, values):
    """Spline coefficients [dim, n3, n2, n1] of a field given by its values at
    the control points of the identity-mapped patch k (Greville collocation,
    direction by direction)."""
    d = prob.dim
    p = int(prob.degree[k])
    ns = prob.n(k)
    C = values.reshape(tuple(ns[::-1]) + (d,))            # [i3][i2][i1][comp]
    C = np.moveaxis(C, -1, 0)                             # [comp][i3][i2][i1]
    for l in range(d):
        kn = spline.open_knots(int(prob.nel[k, l]), p)
        B = spline.basis(kn, p, spline.greville(kn, p))
        axis = d - l                                       # i1 is the last axis
        C = np.moveaxis(np.linalg.solve(B, np.moveaxis(C, axis, 0).reshape(ns[l], -1))
                        .reshape(np.moveaxis(C, axis, 0).shape), 0, axis)
    return C


def polynomial_case(name, amp):
    prob = W.config(name)
    L = [1.0, float(prob.npatch)] + [1.0] * (prob.dim - 2)
    lam, mu = prob.lame[0]
    cu, cf = [], []
    for k in range(prob.npatch):
        X = prob.ctrl[k].reshape(-1, prob.dim)
        cu.append(collocate(prob, k, u_exact(X, amp, L)))
        cf.append(collocate(prob, k, f_exact(X, amp, L, lam, mu)))
    return prob, np.concatenate([c.reshape(-1) for c in cu]), cf


CASES = [("NC-small", np.array([1.0, -0.5])), ("NC3-small", np.array([1.0, -0.5, 0.75]))]


@pytest.mark.parametrize("name,amp", CASES)
def test_nested_rows_hold_for_a_discrete_field(name, amp):
    prob, u, _ = polynomial_case(name, amp)
    s = AFIETI(prob)
    assert np.abs(s.B @ u).max() <= 1e-12 * np.abs(u).max()
    # the same field with the fine copies perturbed violates them
    v = u.copy()
    kc, fc, kf, ff, pf, pc, Wt = s.nested_faces[0]
    i = next(i for i in pf if not s._on_dirichlet(kf, i))
    v[s.dof(kf, 0, i)] += 1e-3
    assert np.abs(s.B @ v).max() > 1e-4


@pytest.mark.parametrize("name,amp", CASES)
def test_nested_direct_and_afieti_reproduce_the_polynomial(name, amp):
    prob, u, cf = polynomial_case(name, amp)
    s = AFIETI(prob)
    f = s.load(cf)
    ud, lamd = s.direct_solve(f)
    assert np.linalg.norm(ud - u) <= 1e-10 * np.linalg.norm(u)
    ui, li, info = s.solve(f, tol=1e-12, maxit=4000)
    assert np.linalg.norm(ui - u) <= 1e-8 * np.linalg.norm(u)
    assert np.linalg.norm(li - lamd) <= 1e-6 * np.linalg.norm(lamd)
    # the multipliers close the torn equations: A u + B^T lambda = f
    A = s.assemble()
    r = f - A @ ud - s.B.T @ lamd
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(f)


def test_nested_counts():
    """Rows: one per copy of a Dirichlet node, m - 1 per free node of m
    copies, one per free fine point of a nested face and component; with the
    constrained space dim Z they add up to the torn dimension."""
    for name in ("NC-small", "NC3-small"):
        s = AFIETI(W.config(name))
        Z = s.conforming_basis()
        assert s.nc + Z.shape[1] == s.ndof
        assert np.linalg.matrix_rank(s.B.toarray()) == s.nc
        nested_rows = sum(len(ids) for (_, _, _, ids) in s.nested_rows)
        free_fine = 0
        for (kc, fc, kf, ff, pf, pc, Wt) in s.nested_faces:
            free_fine += sum(1 for i in pf if not s._on_dirichlet(kf, i))
        assert nested_rows == s.dim * free_fine > 0
