"""Per-patch isogeometric elasticity assembly (Sections 2.2, 3, 4): the spline
geometry map, the stiffness A^(k) of the bilinear form (3.1), the mass M^(k)
and load vectors.  Plain dense quadrature sums over Kronecker-built basis
tables; sizes are meant for the oracle (small patches or a sampled support).
Oracle code: test infrastructure only.

Quadrature reading: Gauss-Legendre with p+1 points per element and direction
(the paper does not state its rule)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import spline


class PatchGeometry:
    """Tables of one patch: knots, quadrature, 1D basis values/derivatives."""

    def __init__(self, ctrl: np.ndarray, p: int, nel):
        self.dim = ctrl.shape[-1]
        self.p = int(p)
        self.nel = [int(x) for x in nel]
        self.ns = [ne + self.p for ne in self.nel]
        self.X = ctrl.reshape(-1, self.dim)                     # [N, d], i1 fastest
        self.knots, self.qx, self.qw, self.T0, self.T1 = [], [], [], [], []
        for ne in self.nel:
            kn = spline.open_knots(ne, self.p)
            x, w, _ = spline.quadrature(kn, self.p)
            self.knots.append(kn)
            self.qx.append(x)
            self.qw.append(w)
            self.T0.append(spline.basis(kn, self.p, x))
            self.T1.append(spline.basis(kn, self.p, x, deriv=1))
        self.nq = [len(x) for x in self.qx]

    # ---- index helpers -------------------------------------------------
    def support_q(self, i_multi):
        """Per-direction quadrature index range covering supp(B_i)."""
        nqe = self.p + 1
        out = []
        for d, i in enumerate(i_multi):
            e_lo = max(0, i - self.p)
            e_hi = min(self.nel[d] - 1, i)
            out.append((e_lo * nqe, (e_hi + 1) * nqe))
        return out

    def neighbour_c(self, i_multi):
        return [(max(0, i - self.p), min(self.ns[d], i + self.p + 1))
                for d, i in enumerate(i_multi)]

    def full_q(self):
        return [(0, n) for n in self.nq]

    def full_c(self):
        return [(0, n) for n in self.ns]

    # ---- tables ----------------------------------------------------------
    def tables(self, qr, cr):
        """Phi_0 and Phi_a (a = parametric derivative direction) restricted to
        quadrature ranges qr and basis ranges cr; rows/cols colex (dir 1 fastest).
        Also returns the tensor-product weights and the column node indices."""
        d = self.dim
        T0 = [self.T0[j][qr[j][0]:qr[j][1], cr[j][0]:cr[j][1]] for j in range(d)]
        T1 = [self.T1[j][qr[j][0]:qr[j][1], cr[j][0]:cr[j][1]] for j in range(d)]
        W = [self.qw[j][qr[j][0]:qr[j][1]] for j in range(d)]

        def kron(tabs):
            out = sp.csr_matrix(np.array([[1.0]]))
            for t in tabs:
                out = sp.kron(sp.csr_matrix(t), out, format="csr")
            return out
        Phi0 = kron(T0)
        Phis = [kron([T1[j] if j == a else T0[j] for j in range(d)]) for a in range(d)]
        w = np.array([1.0])
        for j in range(d):
            w = np.kron(W[j], w)
        # global node indices of the columns
        grids = np.meshgrid(*[np.arange(cr[j][0], cr[j][1]) for j in reversed(range(d))],
                            indexing="ij")
        idx = np.zeros(grids[0].shape, dtype=np.int64)
        stride = 1
        for j in range(d):
            idx += grids[d - 1 - j] * stride
            stride *= self.ns[j]
        return Phi0, Phis, w, idx.reshape(-1)

    def jacobians(self, Phis, cols):
        """J[q, x, a] = d F_x / d eta_a at the quadrature points (isoparametric
        spline map F = sum_i P_i B_i, Section 2.2)."""
        Xc = self.X[cols]
        return np.stack([np.asarray(Ph @ Xc) for Ph in Phis], axis=-1)


def _geometry_block(g: PatchGeometry, qr, cr):
    """Tables plus geometric factors for a sub-block; the columns cr must
    contain every basis function that is non-zero on the quadrature range for
    the Jacobian to be exact, so the Jacobian is evaluated with the full
    support range around qr."""
    d = g.dim
    # basis functions alive on the quadrature range qr
    nqe = g.p + 1
    live = [(qr[j][0] // nqe, min(g.ns[j], (qr[j][1] - 1) // nqe + g.p + 1)) for j in range(d)]
    _, PhisL, _, colsL = g.tables(qr, live)
    J = g.jacobians(PhisL, colsL)
    Phi0, Phis, w, cols = g.tables(qr, cr)
    det = np.linalg.det(J)
    Q = np.linalg.inv(J)                                       # Q[q, a, x] = (J^{-1})_{a x}
    return Phi0, Phis, w, cols, det, Q


def stiffness_block(g: PatchGeometry, lam: float, mu: float, qr=None, cr=None):
    """Dense A over the nodes of range cr, integrated over quadrature range qr:
        A[(l,i),(m,j)] = a(B_i e_l, B_j e_m)
        = int mu (delta_lm grad B_i . grad B_j + d_m B_i d_l B_j)
              + lambda d_l B_i d_m B_j          (eq. 3.1 with eps(u) = sym grad u)
    Returns (A [d*nc, d*nc] component-major, column node indices)."""
    qr = g.full_q() if qr is None else qr
    cr = g.full_c() if cr is None else cr
    d = g.dim
    Phi0, Phis, w, cols, det, Q = _geometry_block(g, qr, cr)
    if np.any(det == 0.0):
        raise ValueError("singular geometry map")
    wd = w * np.abs(det)
    # physical gradients G[x][q, i] = sum_a Q[q, a, x] Phi_a[q, i]
    G = [sum(sp.diags(Q[:, a, x]) @ Phis[a] for a in range(d)).tocsr() for x in range(d)]
    Wd = sp.diags(wd)
    # P[x][y] = int d_x B_i d_y B_j  (quadrature), P[y][x] = P[x][y]^T
    P = [[None] * d for _ in range(d)]
    for x in range(d):
        WGx = (Wd @ G[x]).tocsc()
        for y in range(x, d):
            P[y][x] = (G[y].T @ WGx).toarray()
            if y != x:
                P[x][y] = P[y][x].T
    nc = len(cols)
    A = np.zeros((d * nc, d * nc))
    grad = sum(P[x][x] for x in range(d))
    for l in range(d):
        for m in range(d):
            blk = mu * P[m][l] + lam * P[l][m]
            if l == m:
                blk = blk + mu * grad
            A[l * nc:(l + 1) * nc, m * nc:(m + 1) * nc] = blk
    return A, cols


def stiffness_parts(g: PatchGeometry, qr=None, cr=None):
    """A = lambda * A_lam + mu * A_mu (A^(k) is linear in the Lame values)."""
    A_lam, cols = stiffness_block(g, 1.0, 0.0, qr, cr)
    A_mu, _ = stiffness_block(g, 0.0, 1.0, qr, cr)
    return A_lam, A_mu, cols


def mass_block(g: PatchGeometry, qr=None, cr=None):
    """Scalar mapped mass M_ij = int B_i B_j dx (each component block, eq. 4.8)."""
    qr = g.full_q() if qr is None else qr
    cr = g.full_c() if cr is None else cr
    Phi0, Phis, w, cols, det, Q = _geometry_block(g, qr, cr)
    wd = w * np.abs(det)
    return (Phi0.T @ sp.diags(wd) @ Phi0).toarray(), cols


def stiffness(g: PatchGeometry, lam: float, mu: float) -> np.ndarray:
    A, _ = stiffness_block(g, lam, mu)
    return A


def load_from_coeffs(g: PatchGeometry, c: np.ndarray) -> np.ndarray:
    """f^(k) = M^(k) c for a body force with nodal coefficients c [d, N]."""
    M, _ = mass_block(g)
    return np.concatenate([M @ c[l].reshape(-1) for l in range(g.dim)])


def load_from_function(g: PatchGeometry, fun) -> np.ndarray:
    """f[(l,i)] = int f_l(x) B_i dx for a callable fun(x[Nq, d]) -> [Nq, d]."""
    qr, cr = g.full_q(), g.full_c()
    Phi0, Phis, w, cols, det, Q = _geometry_block(g, qr, cr)
    wd = w * np.abs(det)
    xq = np.asarray(Phi0 @ g.X[cols])
    fv = fun(xq)
    return np.concatenate([Phi0.T @ (wd * fv[:, l]) for l in range(g.dim)])


def min_jacobian(g: PatchGeometry) -> float:
    """Smallest det J over the quadrature points (geometry validity)."""
    _, _, _, _, det, _ = _geometry_block(g, g.full_q(), g.full_c())
    return float(det.min())


def rigid_modes(X: np.ndarray) -> np.ndarray:
    """Rigid body motions evaluated at the control points (Section 4):
    3D: three translations, then (0, x3, -x2), (x3, 0, -x1), (x2, -x1, 0);
    2D: two translations and (x2, -x1).  Returns [d*N, nmodes] component-major;
    isoparametric, so these coefficient vectors represent the motions exactly."""
    N, d = X.shape
    if d == 3:
        x1, x2, x3 = X[:, 0], X[:, 1], X[:, 2]
        z, o = np.zeros(N), np.ones(N)
        cols = [(o, z, z), (z, o, z), (z, z, o), (z, x3, -x2), (x3, z, -x1), (x2, -x1, z)]
    else:
        x1, x2 = X[:, 0], X[:, 1]
        z, o = np.zeros(N), np.ones(N)
        cols = [(o, z), (z, o), (x2, -x1)]
    return np.stack([np.concatenate(c) for c in cols], axis=1)


def sparse_stiffness(g: PatchGeometry, lam: float, mu: float):
    return sp.csr_matrix(stiffness(g, lam, mu))
