"""Fast Diagonalization (Section 5.2.1, Algorithm 1) and the Kronecker-structured
parametric operators of Section 5.2 (the blocks A_hat_l, M_hat_l, their
interior parts).  Oracle code: test infrastructure only.

Axis convention: a patch-component tensor is stored as X[i3, i2, i1] (i1
fastest), so direction l (1-based) is numpy axis d - l.  A Kronecker product
C_d (x) ... (x) C_1 acts on vec(X) as C_l applied along direction l."""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import spline


def gen_eig(K: np.ndarray, M: np.ndarray):
    """Generalised eigendecomposition (eq. 5.8): U^T K U = D, U^T M U = I.
    LAPACK sygv through scipy.linalg.eigh (library step)."""
    D, U = sla.eigh(K, M)
    return D, U


def interior(A: np.ndarray) -> np.ndarray:
    """Drop the first and last index (the interface functions of an open knot
    vector, Section 4)."""
    return A[1:-1, 1:-1]


def coeffs(dim: int, l: int, lam: float, mu: float) -> list:
    """Coefficient of the stiffness term acting in direction j for component l
    (0-based): 2*mu+lambda in direction l, mu elsewhere (Section 5.2)."""
    return [(2.0 * mu + lam) if j == l else mu for j in range(dim)]


def Lambda(D: list, dim: int, l: int, lam: float, mu: float, H: float) -> np.ndarray:
    """Diagonal of Lambda_l (eq. 5.9), shaped [n_d, ..., n_1]:
    H^{d-2} (sum_j c_j D_j + 1)."""
    c = coeffs(dim, l, lam, mu)
    out = np.ones([len(D[j]) for j in reversed(range(dim))])
    for j in range(dim):
        shape = [1] * dim
        shape[dim - 1 - j] = len(D[j])
        out = out + c[j] * np.asarray(D[j]).reshape(shape)
    return (H ** (dim - 2)) * out


def Lambda_interior(Dt: list, dim: int, l: int, lam: float, mu: float) -> np.ndarray:
    """Diagonal of Lambda~_l (eq. 5.10): sum_j c_j D~_j (no mass, no H factor)."""
    c = coeffs(dim, l, lam, mu)
    out = np.zeros([len(Dt[j]) for j in reversed(range(dim))])
    for j in range(dim):
        shape = [1] * dim
        shape[dim - 1 - j] = len(Dt[j])
        out = out + c[j] * np.asarray(Dt[j]).reshape(shape)
    return out


def mode_apply(X: np.ndarray, C: np.ndarray, direction: int, transpose=False) -> np.ndarray:
    """Apply the matrix C (or C^T) along parametric direction `direction`
    (0-based) of the tensor X[i_d, ..., i_1]."""
    dim = X.ndim
    ax = dim - 1 - direction
    Cm = C.T if transpose else C
    Y = np.tensordot(Cm, X, axes=([1], [ax]))          # new axis first
    return np.moveaxis(Y, 0, ax)


def fd_solve(r: np.ndarray, U: list, lam_diag: np.ndarray) -> np.ndarray:
    """Algorithm 1, steps 2-4: r~ = (U_d x...x U_1)^T r, q~ = Lambda^{-1} r~,
    s = (U_d x...x U_1) q~.  r is shaped [n_d, ..., n_1]."""
    dim = r.ndim
    t = r
    for j in range(dim):
        t = mode_apply(t, U[j], j, transpose=True)
    t = t / lam_diag
    for j in range(dim):
        t = mode_apply(t, U[j], j)
    return t


def kron_list(mats: list):
    """C_d (x) ... (x) C_1 for mats = [C_1, ..., C_d] (dense)."""
    out = np.array([[1.0]])
    for C in mats:
        out = np.kron(C, out)
    return out


def A_hat(K: list, M: list, dim: int, l: int, lam: float, mu: float, sparse=False):
    """A_hat_l of Section 5.2: sum over directions j of c_j times the Kronecker
    product with K_j in slot j and M elsewhere.  K, M are lists indexed by
    direction (0-based)."""
    c = coeffs(dim, l, lam, mu)
    kron = (lambda a, b: sp.kron(a, b, format="csr")) if sparse else np.kron
    total = None
    for j in range(dim):
        term = sp.identity(1, format="csr") if sparse else np.array([[1.0]])
        for i in range(dim):
            term = kron(K[i] if i == j else M[i], term)
        term = c[j] * term
        total = term if total is None else total + term
    return total


def M_hat(M: list, dim: int, sparse=False):
    kron = (lambda a, b: sp.kron(a, b, format="csr")) if sparse else np.kron
    out = sp.identity(1, format="csr") if sparse else np.array([[1.0]])
    for i in range(dim):
        out = kron(M[i], out)
    return out


def patch_1d(nel: list, p: int):
    """Univariate K_hat, M_hat per direction for a patch."""
    Ks, Ms = [], []
    for ne in nel:
        K, M = spline.univariate_matrices(int(ne), int(p))
        Ks.append(K)
        Ms.append(M)
    return Ks, Ms


def interior_mask(ns: list) -> np.ndarray:
    """Boolean mask over vec(X) (i1 fastest) of the interior indices, i.e. no
    index on the first/last position in any direction (Section 4)."""
    dim = len(ns)
    grids = np.meshgrid(*[np.arange(n) for n in reversed(ns)], indexing="ij")
    mask = np.ones(grids[0].shape, dtype=bool)
    for j in range(dim):
        g = grids[dim - 1 - j]
        mask &= (g > 0) & (g < ns[j] - 1)
    return mask.reshape(-1)
