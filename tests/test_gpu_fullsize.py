"""Full-size checks at the sizes the benchmark runs (C2, and C4 for the
adjoint), through the C ABI.  The oracle cannot solve these sizes, so the
checks use outputs it can compute one at a time (stiffness and mass rows from
the quadrature over a node's support, single FD blocks, equilibrium rows of
the computed solution) and properties that hold at any size (true residual,
vanishing jumps, gradients against central finite differences)."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import assembly, fd as ofd
from oracle.adjoint import lame_gradient_quadrature

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def node_rows(prob, k, i_multi, x_patch):
    """Oracle rows (A x)_i for the d components of node i of patch k, and the
    mass row (M c)_i, from the quadrature over the node's support."""
    g = assembly.PatchGeometry(prob.ctrl[k], prob.degree[k], prob.nel[k])
    lam, mu = prob.lame[k]
    qr, cr = g.support_q(i_multi), g.neighbour_c(i_multi)
    A, cols = assembly.stiffness_block(g, lam, mu, qr, cr)
    Mm, _ = assembly.mass_block(g, qr, cr)
    node = sum(i_multi[l] * int(np.prod(g.ns[:l])) for l in range(g.dim))
    loc = int(np.where(cols == node)[0][0])
    nc = len(cols)
    d = g.dim
    N = int(np.prod(g.ns))
    xs = np.concatenate([x_patch[l * N + cols] for l in range(d)])
    Ax = np.array([A[l * nc + loc] @ xs for l in range(d)])
    return Ax, Mm[loc], cols, N


@pytest.fixture(scope="module")
def c2():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config("C2")
    s = Solver(prob, prec="fp32", tol=1e-8, use_graph=True)
    yield prob, s
    s.close()


def test_c2_sampled_rows_and_fd_blocks(c2):
    prob, s = c2
    from paper_2001_09626_gb300 import afieti as A
    rng = np.random.default_rng(5)
    coeffs = W.body_force_coeffs(prob)
    f = s.load_vector(coeffs).cpu().numpy()
    x = W.torn_random(prob, 31)[0]
    y = s.apply(A.AFI_OP_STIFFNESS, torch.from_numpy(x).cuda()).cpu().numpy()
    off = prob.offsets()
    for _ in range(12):
        k = int(rng.integers(prob.npatch))
        im = [int(rng.integers(n)) for n in prob.n(k)]
        if _ < 4:   # include patch faces and corners
            im = [0 if rng.random() < 0.5 else n - 1 for n in prob.n(k)]
        Ax, mrow, cols, N = node_rows(prob, k, im, x[off[k]:off[k + 1]])
        node = im[0] + prob.n(k)[0] * (im[1] + prob.n(k)[1] * im[2])
        got = np.array([y[off[k] + l * N + node] for l in range(3)])
        np.testing.assert_allclose(got, Ax, rtol=1e-11, atol=1e-11 * np.abs(Ax).max())
        cf = coeffs[k].reshape(3, -1)
        ref_f = np.array([mrow @ cf[l][cols] for l in range(3)])
        got_f = np.array([f[off[k] + l * N + node] for l in range(3)])
        np.testing.assert_allclose(got_f, ref_f, rtol=1e-12, atol=1e-15)
    # FD blocks at full size, every precision
    r = W.torn_random(prob, 32)[0]
    for prec, tol in (("fp64", 1e-10), ("fp32", 2e-5), ("tf32", 1e-2), ("bf16", 3e-2)):
        s.set_precision(prec)
        out = s.fd(torch.from_numpy(r).cuda()).cpu().numpy()
        for k in (0, 21, 63):
            Ks, Ms = ofd.patch_1d(prob.nel[k], prob.degree[k])
            eig = [ofd.gen_eig(K_, M_) for K_, M_ in zip(Ks, Ms)]
            X = prob.ctrl[k].reshape(-1, 3)
            H = float(np.sqrt(((X.max(0) - X.min(0)) ** 2).sum()))
            ns = prob.n(k)
            N = int(np.prod(ns))
            for l in range(3):
                lamd = ofd.Lambda([e[0] for e in eig], 3, l, prob.lame[k][0], prob.lame[k][1], H)
                a = off[k] + l * N
                ref = ofd.fd_solve(r[a:a + N].reshape(ns[::-1]), [e[1] for e in eig], lamd).reshape(-1)
                err = np.linalg.norm(out[a:a + N] - ref) / np.linalg.norm(ref)
                assert err < tol, (prec, k, l, err)
    s.set_precision("fp32")


def test_c2_solve_properties_and_equilibrium_rows(c2):
    prob, s = c2
    from oracle.ieti import AFIETI
    coeffs = W.body_force_coeffs(prob)
    f = s.load_vector(coeffs)
    u, lam = s.solve(f)
    info = s.last_info
    assert info["relres_true"] <= 1e-8
    orc = AFIETI(prob)          # connectivity and B only (no assembly)
    un = u.cpu().numpy()
    ln = lam.cpu().numpy()
    fn = f.cpu().numpy()
    assert np.linalg.norm(orc.B @ un) <= 1e-7 * np.linalg.norm(un)
    # equilibrium A u + B^T lambda = f on sampled rows, A rows from the oracle
    btl = orc.B.T @ ln
    off = prob.offsets()
    rng = np.random.default_rng(6)
    scale = np.abs(fn).max()
    for _ in range(10):
        k = int(rng.integers(prob.npatch))
        im = [int(rng.integers(n)) for n in prob.n(k)]
        if _ < 5:
            im[int(rng.integers(3))] = 0
        Au, _, _, N = node_rows(prob, k, im, un[off[k]:off[k + 1]])
        node = im[0] + prob.n(k)[0] * (im[1] + prob.n(k)[1] * im[2])
        for l in range(3):
            i = off[k] + l * N + node
            assert abs(fn[i] - Au[l] - btl[i]) <= 1e-6 * scale, (k, im, l)


def stationary_compliance(s, f, u):
    """2 f^T u - u^T A u: equals the compliance f^T u at the exact solution and
    its error is quadratic in the solver error (energy functional)."""
    from paper_2001_09626_gb300 import afieti as A
    Au = s.apply(A.AFI_OP_STIFFNESS, u)
    return float(2.0 * torch.dot(f, u) - torch.dot(u, Au))


def test_c4_adjoint_gradients_against_finite_differences():
    """Compliance J = f^T u on the C4 annulus (72 patches, p = 3, 24^3
    elements): dJ/dtheta from the adjoint (z = u) against the oracle's
    quadrature of -int div u div u / -int 2 eps:eps on sampled patches and
    against central differences (step 1e-6 relative) of the stationary form
    of J evaluated on FP64 solves."""
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config("C4")
    coeffs = W.body_force_coeffs(prob)
    s = Solver(prob, prec="fp64", tol=1e-10, use_graph=True, maxit=6000)
    try:
        f = s.load_vector(coeffs)
        u, _ = s.solve(f)
        z, _ = s.solve_adjoint(f)
        assert (z - u).norm() <= 1e-9 * u.norm()
        grad = s.lame_grad(u, z).cpu().numpy()
        un = u.cpu().numpy()
        off = prob.offsets()
        for k in (0, 35, 71):
            gk = assembly.PatchGeometry(prob.ctrl[k], prob.degree[k], prob.nel[k])
            ref = lame_gradient_quadrature(gk, un[off[k]:off[k + 1]], un[off[k]:off[k + 1]])
            np.testing.assert_allclose(grad[k], ref, rtol=1e-9)
        J0 = float(torch.dot(f, u))
    finally:
        s.close()
    for k, j in ((10, 0), (50, 1)):
        vals = []
        h = 1e-6 * prob.lame[k, j]
        for sgn in (1, -1):
            P2 = W.config("C4")
            P2.lame = prob.lame.copy()
            P2.lame[k, j] += sgn * h
            s2 = Solver(P2, prec="fp64", tol=1e-10, use_graph=True, maxit=6000)
            try:
                f2 = s2.load_vector(coeffs)
                u2, _ = s2.solve(f2)
                vals.append(stationary_compliance(s2, f2, u2))
            finally:
                s2.close()
        fdg = (vals[0] - vals[1]) / (2 * h)
        assert abs(fdg - grad[k, j]) <= 1e-5 * abs(grad[k, j]), (k, j, fdg, grad[k, j], J0)
