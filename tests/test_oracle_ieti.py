"""Pins for the oracle's AF-IETI (Section 4, Section 5.2, Remark 1): the
constraint count against dim of the conforming space, full row rank and the
block-diagonal B B^T, the projector identities, lambda_0, the iterative
solution against the conforming direct solve (the unique solution of
eq. 4.5), vanishing jumps, the monotone MINRES estimate and MINRES against a
dense solve; plus the adjoint gradients against central finite differences."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import adjoint
from oracle.ieti import AFIETI
from oracle.minres import minres


@pytest.fixture(scope="module")
def c1():
    P = W.config("C1")
    s = AFIETI(P)
    f = s.load(W.body_force_coeffs(P))
    return P, s, f


@pytest.fixture(scope="module")
def c2s():
    P = W.config("C2-small")
    s = AFIETI(P)
    f = s.load(W.body_force_coeffs(P))
    return P, s, f


def test_constraint_counts(c1, c2s):
    for P, s, _ in (c1, c2s):
        Z = s.conforming_basis()
        assert s.nc == s.ndof - Z.shape[1]
    assert c1[1].nc == 222                     # 152 Dirichlet + 64 edge + 6 cross-point rows


def test_B_rank_and_BBt_blocks(c1):
    _, s, _ = c1
    Bd = s.B.toarray()
    assert np.linalg.matrix_rank(Bd) == s.nc
    BBt = s.BBt.toarray()
    seen = np.zeros(s.nc, dtype=bool)
    for c, n, ids in s.node_rows:
        if not ids:
            continue
        blk = BBt[np.ix_(ids, ids)]
        m = len(ids)
        ref = np.eye(m) if s.dirichlet[n] else np.eye(m) + np.ones((m, m))
        np.testing.assert_array_equal(blk, ref)
        seen[ids] = True
        others = np.setdiff1d(np.arange(s.nc), ids)
        assert not BBt[np.ix_(ids, others)].any()
    assert seen.all()


def test_projectors(c2s):
    _, s, f = c2s
    rng = np.random.default_rng(7)
    x = rng.standard_normal(s.nc)
    y = rng.standard_normal(s.nc)
    px = s.P_chi(x)
    np.testing.assert_allclose(s.P_chi(px), px, atol=1e-10)
    np.testing.assert_allclose(s.G.T @ px, 0.0, atol=1e-10)
    assert abs(px @ y - x @ s.P_chi(y)) < 1e-9
    Rd = s.R.toarray()
    for j in range(0, Rd.shape[1], 5):
        np.testing.assert_allclose(s.P_u(Rd[:, j]), 0.0, atol=1e-11)
    lam0 = s.lambda0(f)
    np.testing.assert_allclose(s.G.T @ lam0, s.R.T @ f, atol=1e-11)


@pytest.mark.parametrize("which", ["c1", "c2s"])
def test_afieti_equals_direct(which, request):
    _, s, f = request.getfixturevalue(which)
    u, lam, info = s.solve(f, tol=1e-8)
    ud, ld = s.direct_solve(f)
    assert info["true_relres"] <= 1e-8
    assert np.linalg.norm(u - ud) <= 1e-6 * np.linalg.norm(ud)
    assert np.linalg.norm(lam - ld) <= 1e-6 * np.linalg.norm(ld)
    assert np.linalg.norm(s.B @ u) <= 1e-8 * np.linalg.norm(u)
    h = np.array(info["history"])
    assert (np.diff(h) <= 1e-12).all()        # MINRES residual estimate is monotone


@pytest.mark.parametrize("name,faces", [("C2-small", (0, 1)), ("C1", (0, 1))])
def test_neumann_faces(name, faces):
    """Outer faces with the natural condition (the x-faces, as in the paper's
    weak-scaling test): fewer constraint rows, the same identities, AF-IETI
    equals the conforming direct solve, and the solution vanishes exactly on
    the Dirichlet nodes but not on the free faces."""
    P = W.with_neumann(W.config(name), faces)
    s = AFIETI(P)
    Pd = W.config(name)
    sd = AFIETI(Pd)
    assert s.nc < sd.nc
    Z = s.conforming_basis()
    assert s.nc == s.ndof - Z.shape[1]
    f = s.load(W.body_force_coeffs(P))
    u, lam, info = s.solve(f, tol=1e-10)
    ud, ld = s.direct_solve(f)
    assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)
    assert np.linalg.norm(s.B @ u) <= 1e-9 * np.linalg.norm(u)
    on_free, on_dir = [], []
    for k in range(P.npatch):
        g = s.geo[k]
        for l in range(P.dim):
            for idx in np.ndindex(*g.ns[::-1]):
                i = idx[::-1]
                node = int(np.ravel_multi_index(idx, g.ns[::-1]))
                dof = s.dof(k, l, node)
                if P.dirichlet_face[k, 2] and i[1] == 0:       # y = 0 face: Dirichlet
                    on_dir.append(dof)
                if not P.dirichlet_face[k, 0] and Pd.dirichlet_face[k, 0] and i[0] == 0 \
                        and 0 < i[1] < g.ns[1] - 1:             # free x = 0 face, off the edges
                    on_free.append(dof)
    assert np.all(u[on_dir] == 0.0) or np.max(np.abs(u[on_dir])) <= 1e-10 * np.max(np.abs(u))
    assert np.max(np.abs(u[on_free])) > 1e-3 * np.max(np.abs(u))


def test_preconditioner_spd_on_subspace():
    P = W.config("C1-small")
    s = AFIETI(P)
    n, m = s.ndof, s.nc
    # basis of range(A) x ker(G^T) through the projectors
    E = np.eye(n + m)
    M = np.stack([np.concatenate(s.precond_apply(E[i, :n], E[i, n:])) for i in range(n + m)], axis=1)
    np.testing.assert_allclose(M, M.T, atol=1e-9 * abs(M).max())
    ev = np.linalg.eigvalsh(0.5 * (M + M.T))
    assert ev.min() > -1e-9 * ev.max()


def test_minres_matches_dense_solve():
    rng = np.random.default_rng(11)
    n = 60
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.concatenate([rng.uniform(1, 5, 40), -rng.uniform(1, 5, 20)])) @ Q.T
    L = rng.standard_normal((n, n)) / np.sqrt(n)
    Minv = L @ L.T + np.eye(n)
    b = rng.standard_normal(n)
    x, info = minres(lambda v: A @ v, b, lambda v: Minv @ v, tol=1e-12, maxit=500)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-10)
    assert (np.diff(info["history"]) <= 1e-14).all()


def test_adjoint_gradients_vs_finite_differences():
    P = W.config("C1-small")
    P.lame = P.lame * np.array([[1.0, 1.0], [1.3, 0.8], [0.7, 1.1], [1.0, 1.2]])
    s = AFIETI(P)
    f = s.load(W.body_force_coeffs(P))
    J, dJdf, dJdlame = adjoint.compliance_and_grads(s, f)
    u, _, _ = s.solve(f, tol=1e-12)
    J_it, _, g_it = adjoint.compliance_and_grads(s, f, direct=False)
    np.testing.assert_allclose(g_it, dJdlame, rtol=1e-7)
    h = 1e-6
    for k in range(P.npatch):
        for j in range(2):
            vals = []
            for sgn in (1, -1):
                P2 = W.config("C1-small")
                P2.lame = P.lame.copy()
                P2.lame[k, j] += sgn * h
                s2 = AFIETI(P2)
                u2, _ = s2.direct_solve(f)
                vals.append(f @ u2)
            fdg = (vals[0] - vals[1]) / (2 * h)
            assert abs(fdg - dJdlame[k, j]) <= 1e-5 * max(abs(fdg), 1e-12), (k, j, fdg, dJdlame[k, j])
    rng = np.random.default_rng(2)
    for i in rng.choice(s.ndof, 5, replace=False):
        e = np.zeros(s.ndof); e[i] = h
        up, _ = s.direct_solve(f + e)
        um, _ = s.direct_solve(f - e)
        fdg = ((f + e) @ up - (f - e) @ um) / (2 * h)
        assert abs(fdg - dJdf[i]) <= 1e-5 * max(abs(fdg), 1e-8)


def test_lame_gradient_quadrature_equals_matrix_form():
    """-int div z div u and -int 2 eps(z):eps(u) by quadrature equal
    -z^T A_lam u and -z^T A_mu u from the assembled blocks."""
    from oracle import adjoint
    for name in ("C1-small", "C2-small"):
        P = W.config(name)
        s = AFIETI(P)
        rng = np.random.default_rng(9)
        u = rng.standard_normal(s.ndof)
        z = rng.standard_normal(s.ndof)
        ref = adjoint.lame_gradient(s, u, z)
        for k in range(P.npatch):
            sl = slice(s.off[k], s.off[k + 1])
            q = adjoint.lame_gradient_quadrature(s.geo[k], u[sl], z[sl])
            np.testing.assert_allclose(q, ref[k], rtol=1e-11, atol=1e-13)


def test_exact_local_solvers():
    """Section 5.1: S^(k) by harmonic extension equals the dense Schur
    complement A_GG - A_GI A_II^{-1} A_IG, maps the shell traces of the rigid
    modes to zero, is symmetric; P_A^ex^{-1} inverts A + H^{-2} M; and AF-IETI
    with the exact local solvers equals the direct solve in fewer iterations
    than with the inexact ones (the paper's tables)."""
    from oracle import assembly, fd as ofd
    import scipy.sparse as sp
    P = W.config("C1-small")
    s = AFIETI(P, precond="exact")
    A = s.assemble()
    rng = np.random.default_rng(31)
    for k, g in enumerate(s.geo):
        sl = slice(s.off[k], s.off[k + 1])
        Ak = A[sl][:, sl].toarray()
        inner = np.tile(ofd.interior_mask(g.ns), s.dim)
        G, I = ~inner, inner
        Sd = Ak[np.ix_(G, G)] - Ak[np.ix_(G, I)] @ np.linalg.solve(Ak[np.ix_(I, I)], Ak[np.ix_(I, G)])
        t = np.zeros(s.ndof)
        tk = rng.standard_normal(int(G.sum()))
        t[s.off[k] + np.nonzero(G)[0]] = tk
        y = s.S_exact(t)[sl]
        np.testing.assert_allclose(y[G], Sd @ tk, rtol=1e-10, atol=1e-12 * np.abs(Sd).max())
        assert not y[I].any()
        np.testing.assert_allclose(Sd, Sd.T, atol=1e-12 * np.abs(Sd).max())
        Mk, _ = assembly.mass_block(g)
        K = Ak + np.kron(np.eye(s.dim), Mk) / s.H[k] ** 2
        x = rng.standard_normal(K.shape[0])
        r = np.zeros(s.ndof)
        r[sl] = K @ x
        np.testing.assert_allclose(s.PA_inv_exact(r)[sl], x, rtol=1e-10, atol=1e-12)
    Rd = s.R.toarray()
    for j in range(Rd.shape[1]):
        t = Rd[:, j] * s.shell
        assert np.linalg.norm(s.S_exact(t)) <= 1e-12 * np.linalg.norm(t)
    for name in ("C1-small", "C1"):
        P = W.config(name)
        se, si = AFIETI(P, precond="exact"), AFIETI(P)
        f = se.load(W.body_force_coeffs(P))
        u, lam, info = se.solve(f, tol=1e-10)
        _, _, info_i = si.solve(f, tol=1e-10)
        ud, ld = se.direct_solve(f)
        assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)
        assert info["iters"] < info_i["iters"]


def test_inexact_schur_pins():
    """eqs. 5.4-5.5, 5.7: S_hat by harmonic extension equals the dense Schur
    complement H^{d-2} (A_GG - A_GI A_II^{-1} A_IG) of the parametric A_hat_l,
    maps constant shell vectors to zero (A_hat has the constants in its kernel),
    and P_S is symmetric positive semi-definite."""
    from oracle import fd as ofd
    for name in ("C1-small", "C2-small"):
        P = W.config(name)
        s = AFIETI(P)
        rng = np.random.default_rng(51)
        for k, g in enumerate(s.geo[:2]):
            lam, mu = P.lame[k]
            Ks, Ms = ofd.patch_1d(g.nel, g.p)
            inner = ofd.interior_mask(g.ns)
            G, I = ~inner, inner
            Hs = s.H[k] ** (s.dim - 2)
            for l in range(s.dim):
                Ah = ofd.A_hat(Ks, Ms, s.dim, l, lam, mu)
                Sd = Hs * (Ah[np.ix_(G, G)] - Ah[np.ix_(G, I)] @ np.linalg.solve(Ah[np.ix_(I, I)], Ah[np.ix_(I, G)]))
                t = np.zeros(s.ndof)
                base = s.dof(k, l, 0)
                tk = rng.standard_normal(int(G.sum()))
                t[base + np.nonzero(G)[0]] = tk
                y = s.S_hat_H(t)[base:base + s.N[k]]
                np.testing.assert_allclose(y[G], Sd @ tk, rtol=1e-9, atol=1e-11 * np.abs(Sd).max())
                assert not y[I].any()
                one = np.zeros(s.ndof)
                one[base + np.nonzero(G)[0]] = 1.0
                assert np.abs(s.S_hat_H(one)).max() <= 1e-11 * np.abs(Sd).max()
        x, y = rng.standard_normal(s.nc), rng.standard_normal(s.nc)
        assert abs(x @ s.P_S(y) - y @ s.P_S(x)) <= 1e-10 * np.linalg.norm(x) * np.linalg.norm(s.P_S(y))
        assert x @ s.P_S(x) >= -1e-12 * np.linalg.norm(x) ** 2
