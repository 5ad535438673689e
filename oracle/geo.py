"""Geometry-inclusion local solvers (Section 5.2.3): the Kronecker-structured
blocks A~_l, M~_l built from separable approximations of the diagonal of the
elasticity coefficient, the diagonal scalings D_A, D_S, and the resulting
P~_A^inex (eq. 5.12) and S~ (eq. 5.13).  Oracle code: test infrastructure only.

For component l the stiffness block is int grad B_i^T C_l grad B_j over the
parametric domain with
    C_l = [mu J^{-1} J^{-T} + (mu + lambda) J^{-1} e_l e_l^T J^{-T}] |det J|,
and every diagonal entry is replaced by a product of univariate factors,
    [C_l]_ii ~ nu_{l,i}(eta_i) prod_{j != i} beta_{l,j}(eta_j).

Readings (the paper cites the approximation algorithm, a variant of
Wachspress's and Diliberto-Straus's, without stating it):
  * the fit is made in the logarithm, where the products become sums of
    univariate functions, at the Gauss points of the assembly;
  * besides the d diagonal entries, the shared factors must also fit the mass
    coefficient, |det J| ~ prod_j beta_{l,j}(eta_j): the paper builds the
    modified mass M~_l from the same beta_{l,j}, and this fixes the scaling
    freedom between the nu and beta factors;
  * the fit uses Diliberto-Straus sweeps (best uniform approximation by sums
    of univariate functions): each factor in turn is set to the mid-range
    (max + min) / 2 of its current residual over the other variables, a shared
    factor over all the targets it enters, until no factor moves by more than
    1e-14 (at most 500 sweeps).  A separable coefficient is reproduced exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fd


def coefficient_diagonals(g, lam: float, mu: float, l: int):
    """The d diagonal entries of C_l and |det J| at the Gauss points, each as an
    array indexed [q_1, ..., q_d] (direction j along axis j)."""
    d = g.dim
    Phi0, Phis, w, cols = g.tables(g.full_q(), g.full_c())
    J = g.jacobians(Phis, cols)                       # J[q, x, a] = dF_x / d eta_a
    Q = np.linalg.inv(J)                              # Q[q, a, x] = (J^{-1})_{a x}
    det = np.abs(np.linalg.det(J))
    shape_rev = [g.nq[j] for j in reversed(range(d))]   # flat q has q_1 fastest

    def grid(v):
        return np.transpose(v.reshape(shape_rev))       # -> [q_1, ..., q_d]
    diag = []
    for a in range(d):
        c = (mu * (Q[:, a, :] ** 2).sum(axis=1) + (mu + lam) * Q[:, a, l] ** 2) * det
        diag.append(grid(c))
    return diag, grid(det)


def _others(arr, axis):
    return tuple(j for j in range(arr.ndim) if j != axis)


def separable_fit(diag, det, sweeps=500, tol=1e-14):
    """Univariate factors nu_i, beta_j (lists of 1D arrays over the Gauss
    points of each direction) with diag[i] ~ nu_i prod_{j != i} beta_j and
    det ~ prod_j beta_j, by Diliberto-Straus mid-range sweeps in the logarithm."""
    d = det.ndim
    Li = [np.log(x) for x in diag]
    L0 = np.log(det)
    a = [np.zeros(det.shape[i]) for i in range(d)]    # log nu_i
    b = [np.zeros(det.shape[j]) for j in range(d)]    # log beta_j

    def along(v, axis):
        shape = [1] * d
        shape[axis] = len(v)
        return v.reshape(shape)

    def bsum(skip):
        s = np.zeros(det.shape)
        for j in range(d):
            if j not in skip:
                s = s + along(b[j], j)
        return s
    for _ in range(sweeps):
        move = 0.0
        for i in range(d):
            R = Li[i] - bsum({i})
            new = 0.5 * (R.max(axis=_others(R, i)) + R.min(axis=_others(R, i)))
            move = max(move, np.abs(new - a[i]).max())
            a[i] = new
        for j in range(d):
            # targets containing beta_j: the mass coefficient and the entries i != j
            res = [L0 - bsum({j})]
            for i in range(d):
                if i != j:
                    res.append(Li[i] - along(a[i], i) - bsum({i, j}))
            hi = np.max([r.max(axis=_others(r, j)) for r in res], axis=0)
            lo = np.min([r.min(axis=_others(r, j)) for r in res], axis=0)
            new = 0.5 * (hi + lo)
            move = max(move, np.abs(new - b[j]).max())
            b[j] = new
        if move <= tol:
            break
    return [np.exp(x) for x in a], [np.exp(x) for x in b]


def univariate(g, nu, beta):
    """K~_m = int nu_m b_i' b_j', M~_m = int beta_m b_i b_j per direction m."""
    K, M = [], []
    for m in range(g.dim):
        w = g.qw[m]
        K.append(g.T1[m].T @ np.diag(w * nu[m]) @ g.T1[m])
        M.append(g.T0[m].T @ np.diag(w * beta[m]) @ g.T0[m])
    return K, M


def kron_terms(K, M):
    """A~ = sum_m (K in slot m, M elsewhere) and M~ = M_d x ... x M_1 (sparse)."""
    d = len(K)
    A = None
    for m in range(d):
        t = sp.identity(1, format="csr")
        for j in range(d):
            t = sp.kron(sp.csr_matrix(K[j] if j == m else M[j]), t, format="csr")
        A = t if A is None else A + t
    Mt = sp.identity(1, format="csr")
    for j in range(d):
        Mt = sp.kron(sp.csr_matrix(M[j]), Mt, format="csr")
    return A.tocsr(), Mt.tocsr()


class GeoLocal:
    """Per patch and component: A~_l, M~_l, the scalings and factorisations of
    P~_A^{inex,(k)} (eq. 5.12) and of (A~_l)_II for S~ (eq. 5.13)."""

    def __init__(self, g, lam, mu, H, A_patch, M_scalar):
        d = g.dim
        N = int(np.prod(g.ns))
        self.mask = fd.interior_mask(g.ns)
        self.per = []
        for l in range(d):
            diag, det = coefficient_diagonals(g, lam, mu, l)
            nu, beta = separable_fit(diag, det)
            K, M = univariate(g, nu, beta)
            At, Mt = kron_terms(K, M)
            All = A_patch[l * N:(l + 1) * N, l * N:(l + 1) * N]
            P = At + Mt / H ** 2
            DA = (All.diagonal() + M_scalar.diagonal() / H ** 2) / P.diagonal()
            DS = All.diagonal() / At.diagonal()
            self.per.append(dict(At=At, Mt=Mt, K=K, M=M, nu=nu, beta=beta, DA=DA, DS=DS,
                                 P=spla.splu(P.tocsc()),
                                 AII=spla.splu(At[self.mask][:, self.mask].tocsc())))

    def PA_inv(self, l, r):
        """P~_A^{-1} r for component l: D_A^{-1/2} (A~ + H^{-2} M~)^{-1} D_A^{-1/2} r."""
        q = self.per[l]
        s = 1.0 / np.sqrt(q["DA"])
        return s * q["P"].solve(s * r)

    def S(self, l, t):
        """D_S^{1/2} S~_l D_S^{1/2} t on the shell (zero in the interior): the
        Schur complement of A~_l with the interior eliminated."""
        q = self.per[l]
        mask = self.mask
        v = np.where(mask, 0.0, np.sqrt(q["DS"]) * t)
        y = q["At"] @ v
        v[mask] = -q["AII"].solve(y[mask])
        z = q["At"] @ v
        return np.where(mask, 0.0, np.sqrt(q["DS"]) * z)
