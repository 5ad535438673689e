"""Pins for the oracle's patch assembly (Sections 2.2, 3, 4): rigid modes in
the kernel (isoparametric, Section 4), symmetry and rank, the closed-form
energy of a constant strain, the Kronecker special case on axis-aligned boxes
(A_ll = a^{d-2} A_hat_l, off-diagonal blocks from 1D b'b integrals, mass
a^d M_3 x M_2 x M_1) and the O(h^{p+1}) L2 convergence of a manufactured
solution."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import assembly, fd, spline
from oracle.ieti import AFIETI

LAM, MU = 0.3 / 0.52, 1.0 / 2.6


def box_patch(nels, p, side=1.0, affine=None):
    d = len(nels)
    g = [spline.greville(spline.open_knots(ne, p), p) for ne in nels]
    mesh = np.meshgrid(*g[::-1], indexing="ij")
    X = side * np.stack(mesh[::-1], axis=-1)
    if affine is not None:
        X = X @ np.asarray(affine).T
    return assembly.PatchGeometry(X, p, nels)


def patches_from(name):
    P = W.config(name)
    return [(assembly.PatchGeometry(P.ctrl[k], P.degree[k], P.nel[k]), P.lame[k])
            for k in range(P.npatch)]


@pytest.mark.parametrize("name,which", [("C2-small", [0, 7]), ("C4-small", [0, 5]),
                                        ("C5-small", [3]), ("C1-small", [0, 3])])
def test_rigid_modes_in_kernel_symmetric_rank(name, which):
    pats = patches_from(name)
    for k in which:
        g, (lam, mu) = pats[k]
        A = assembly.stiffness(g, lam, mu)
        np.testing.assert_allclose(A, A.T, atol=1e-12 * abs(A).max())
        R = assembly.rigid_modes(g.X)
        np.testing.assert_allclose(A @ R, 0.0, atol=1e-10 * abs(A).max() * abs(R).max())
        ev = np.linalg.eigvalsh(A)
        nm = R.shape[1]
        assert abs(ev[:nm]).max() < 1e-10 * ev[-1]
        assert ev[nm] > 1e-6 * ev[-1]


@pytest.mark.parametrize("dim,affine", [(3, None), (3, [[1.0, 0.3, 0.0], [0.1, 0.9, 0.2], [0.0, -0.2, 1.3]]),
                                        (2, [[1.2, 0.4], [-0.1, 0.8]])])
def test_constant_strain_energy(dim, affine):
    nels = [3, 2, 4][:dim]
    g = box_patch(nels, 2, side=0.7, affine=affine)
    eps = np.array([[0.3, 0.1, -0.2], [0.1, -0.4, 0.05], [-0.2, 0.05, 0.25]])[:dim, :dim]
    rot = np.array([[0, 0.7, -0.1], [-0.7, 0, 0.3], [0.1, -0.3, 0]])[:dim, :dim]
    u = (g.X @ (eps + rot).T).T.reshape(-1)       # linear field, rigid part added
    A = assembly.stiffness(g, LAM, MU)
    vol = 0.7 ** dim * (abs(np.linalg.det(affine)) if affine is not None else 1.0)
    exact = vol * (2 * MU * np.sum(eps * eps) + LAM * np.trace(eps) ** 2)
    assert abs(u @ A @ u - exact) < 1e-11 * exact


@pytest.mark.parametrize("nels,p,a", [([3, 2, 4], 2, 0.5), ([2, 3, 2], 3, 1.7), ([4, 3], 2, 0.3)])
def test_box_kronecker_special_case(nels, p, a):
    d = len(nels)
    g = box_patch(nels, p, side=a)
    A = assembly.stiffness(g, LAM, MU)
    Ks, Ms = fd.patch_1d(nels, p)
    Cs = []
    for ne in nels:
        kn = spline.open_knots(ne, p)
        x, w, _ = spline.quadrature(kn, p)
        Cs.append(spline.basis(kn, p, x, 1).T @ (w[:, None] * spline.basis(kn, p, x)))
    N = int(np.prod([ne + p for ne in nels]))
    for l in range(d):
        blk = A[l * N:(l + 1) * N, l * N:(l + 1) * N]
        np.testing.assert_allclose(blk, a ** (d - 2) * fd.A_hat(Ks, Ms, d, l, LAM, MU),
                                   atol=1e-11 * abs(blk).max())
        for m in range(d):
            if m == l:
                continue
            t1 = fd.kron_list([Cs[j] if j == m else (Cs[j].T if j == l else Ms[j]) for j in range(d)])
            t2 = fd.kron_list([Cs[j] if j == l else (Cs[j].T if j == m else Ms[j]) for j in range(d)])
            ref = a ** (d - 2) * (MU * t1 + LAM * t2)
            blk = A[l * N:(l + 1) * N, m * N:(m + 1) * N]
            np.testing.assert_allclose(blk, ref, atol=1e-11 * abs(A).max())
    Mm, _ = assembly.mass_block(g)
    np.testing.assert_allclose(Mm, a ** d * fd.M_hat(Ms, d), atol=1e-14)


def _manufactured_2d():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    u = [sympy.sin(sympy.pi * x) * sympy.sin(sympy.pi * y),
         sympy.sin(sympy.pi * x) * sympy.sin(2 * sympy.pi * y) * (1 + x)]
    X = [x, y]
    eps = [[(sympy.diff(u[i], X[j]) + sympy.diff(u[j], X[i])) / 2 for j in range(2)] for i in range(2)]
    tr = eps[0][0] + eps[1][1]
    sig = [[2 * MU * eps[i][j] + (LAM * tr if i == j else 0) for j in range(2)] for i in range(2)]
    f = [-sum(sympy.diff(sig[i][j], X[j]) for j in range(2)) for i in range(2)]
    uf = sympy.lambdify((x, y), u, "numpy")
    ff = sympy.lambdify((x, y), f, "numpy")
    return (lambda q: np.stack(np.broadcast_arrays(*uf(q[:, 0], q[:, 1])), axis=1),
            lambda q: np.stack(np.broadcast_arrays(*ff(q[:, 0], q[:, 1])), axis=1))


def test_manufactured_solution_l2_rate():
    """Homogeneous-Dirichlet manufactured field on the unit square (2x2 patches,
    p = 2): the L2 error of the conforming Galerkin solution decays like
    h^{p+1}."""
    uex, fex = _manufactured_2d()
    p = 2
    errs = []
    for nel in (4, 8, 16):
        P = W.unit_box(2, (2, 2), p, nel)
        s = AFIETI(P)
        f = np.concatenate([assembly.load_from_function(g, fex) for g in s.geo])
        u, _ = s.direct_solve(f)
        e2 = 0.0
        for k, g in enumerate(s.geo):
            Phi0, _, w, cols, det, _ = assembly._geometry_block(g, g.full_q(), g.full_c())
            xq = np.asarray(Phi0 @ g.X[cols])
            uk = u[s.off[k]:s.off[k + 1]].reshape(2, -1)
            uh = np.stack([Phi0 @ uk[0], Phi0 @ uk[1]], axis=1)
            e2 += np.sum(w * abs(det) * np.sum((uh - uex(xq)) ** 2, axis=1))
        errs.append(np.sqrt(e2))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 1 - 0.3, (errs, rates)


@pytest.mark.parametrize("name", ["C2-small", "C2-mid"])
def test_jittered_geometry_is_valid(name):
    """Interior jitter of 10% of the element size keeps det J well positive
    (the map stays a valid parametrisation, Section 2.2)."""
    P = W.config(name)
    for k in range(P.npatch):
        g = assembly.PatchGeometry(P.ctrl[k], P.degree[k], P.nel[k])
        side = 1.0 / P.grid[0]
        assert assembly.min_jacobian(g) > 0.5 * side ** 3
