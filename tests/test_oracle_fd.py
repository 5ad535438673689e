"""Pins for the oracle's Fast Diagonalization (Algorithm 1, eqs. 5.8-5.10):
the generalised eigen identities, the FD solve against a dense direct solve of
the Kronecker-sum system on small patches (3D and 2D, every component),
invariance to eigenvector signs and the interior variant."""
import numpy as np
import pytest

from oracle import fd

LAM, MU = 0.3 / 0.52, 1.0 / 2.6


@pytest.mark.parametrize("p,nel", [(2, 3), (3, 5), (4, 4), (5, 2)])
def test_eigen_identities(p, nel):
    Ks, Ms = fd.patch_1d([nel], p)
    K, M = Ks[0], Ms[0]
    D, U = fd.gen_eig(K, M)
    np.testing.assert_allclose(U.T @ M @ U, np.eye(len(D)), atol=1e-12)
    np.testing.assert_allclose(U.T @ K @ U, np.diag(D), atol=1e-9 * D.max())
    assert abs(D.min()) < 1e-9 * D.max()
    v = U[:, np.argmin(D)]
    np.testing.assert_allclose(v / v[0], np.ones_like(v), atol=1e-8)
    # interior pencil is definite
    Dt, Ut = fd.gen_eig(fd.interior(K), fd.interior(M))
    assert Dt.min() > 0
    np.testing.assert_allclose(Ut.T @ fd.interior(M) @ Ut, np.eye(len(Dt)), atol=1e-12)


def _setup(nels, p):
    Ks, Ms = fd.patch_1d(nels, p)
    eig = [fd.gen_eig(K, M) for K, M in zip(Ks, Ms)]
    return Ks, Ms, [e[0] for e in eig], [e[1] for e in eig]


@pytest.mark.parametrize("nels,p,H", [([2, 3, 4], 2, 0.7), ([3, 3, 3], 3, 1.3), ([4, 2], 2, 0.5),
                                      ([3, 5], 3, 2.0)])
def test_fd_equals_dense_kronecker_solve(nels, p, H):
    dim = len(nels)
    Ks, Ms, D, U = _setup(nels, p)
    ns = [ne + p for ne in nels]
    rng = np.random.default_rng(3)
    for l in range(dim):
        P = H ** (dim - 2) * (fd.A_hat(Ks, Ms, dim, l, LAM, MU) + fd.M_hat(Ms, dim))
        r = rng.standard_normal(int(np.prod(ns)))
        s_dense = np.linalg.solve(P, r)
        lam = fd.Lambda(D, dim, l, LAM, MU, H)
        s = fd.fd_solve(r.reshape(ns[::-1]), U, lam).reshape(-1)
        np.testing.assert_allclose(s, s_dense, rtol=1e-10, atol=1e-12 * abs(s_dense).max())
        # FD(P r) = r
        back = fd.fd_solve((P @ r).reshape(ns[::-1]), U, lam).reshape(-1)
        np.testing.assert_allclose(back, r, atol=1e-9)
        # Lambda is the diagonalised operator, eq. 5.9
        Uk = fd.kron_list(U)
        np.testing.assert_allclose(Uk.T @ P @ Uk, np.diag(lam.reshape(-1)),
                                   atol=1e-9 * lam.max())


def test_fd_sign_invariance():
    nels, p, H = [3, 4, 2], 3, 1.0
    Ks, Ms, D, U = _setup(nels, p)
    ns = [ne + p for ne in nels]
    r = np.random.default_rng(4).standard_normal(ns[::-1])
    lam = fd.Lambda(D, 3, 1, LAM, MU, H)
    s0 = fd.fd_solve(r, U, lam)
    flips = [u * np.where(np.arange(u.shape[1]) % 2 == 0, -1.0, 1.0) for u in U]
    s1 = fd.fd_solve(r, flips, lam)
    np.testing.assert_allclose(s0, s1, atol=1e-12)


@pytest.mark.parametrize("nels,p", [([3, 4, 3], 2), ([4, 4, 4], 3), ([3, 4], 2)])
def test_interior_fd_equals_dense(nels, p):
    dim = len(nels)
    Ks, Ms = fd.patch_1d(nels, p)
    ns = [ne + p for ne in nels]
    mask = fd.interior_mask(ns)
    eig = [fd.gen_eig(fd.interior(K), fd.interior(M)) for K, M in zip(Ks, Ms)]
    Dt, Ut = [e[0] for e in eig], [e[1] for e in eig]
    rng = np.random.default_rng(5)
    for l in range(dim):
        A = fd.A_hat(Ks, Ms, dim, l, LAM, MU)
        AII = A[mask][:, mask]
        r = rng.standard_normal(AII.shape[0])
        lam = fd.Lambda_interior(Dt, dim, l, LAM, MU)
        s = fd.fd_solve(r.reshape([n - 2 for n in ns][::-1]), Ut, lam).reshape(-1)
        np.testing.assert_allclose(s, np.linalg.solve(AII, r), rtol=1e-9, atol=1e-12)


def test_a_hat_singular_with_constants_in_kernel():
    """A_hat_l is singular (all-DoF 1D stiffness), constants are in its kernel."""
    Ks, Ms = fd.patch_1d([3, 2, 4], 2)
    A = fd.A_hat(Ks, Ms, 3, 0, LAM, MU)
    np.testing.assert_allclose(A @ np.ones(A.shape[0]), 0.0, atol=1e-11)
