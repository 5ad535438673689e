"""The remaining full-size configurations, through the C ABI.

C3: quarter annulus, 6x4x3 patches with per-column element counts and p = 4
(uneven tensors, some too large for the single-CTA tensor-core FD, which then
run on the three-pass tensor-core kernels): full TF32 solve to 1e-8 with sampled oracle
stiffness rows and equilibrium rows, vanishing jumps, sampled FD blocks.
C5: twisted box, 8x8x4 patches, p = 4, 48^3 elements (108 M DoF per
right-hand side; its stencil would need 1.9 TB): a local-solvers-only
context, FD on two right-hand sides in one call, sampled blocks against the
oracle's Algorithm 1."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import fd as ofd

from test_gpu_fullsize import node_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def fd_block_ref(prob, k, l, r_block):
    Ks, Ms = ofd.patch_1d(prob.nel[k], prob.degree[k])
    eig = [ofd.gen_eig(K, M) for K, M in zip(Ks, Ms)]
    X = prob.ctrl[k].reshape(-1, 3)
    H = float(np.sqrt(((X.max(0) - X.min(0)) ** 2).sum()))
    lamd = ofd.Lambda([e[0] for e in eig], 3, l, prob.lame[k][0], prob.lame[k][1], H)
    ns = prob.n(k)
    return ofd.fd_solve(r_block.reshape(ns[::-1]), [e[1] for e in eig], lamd).reshape(-1)


def test_c3_uneven_solve_and_samples():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    from paper_2001_09626_gb300 import afieti as A
    from oracle.ieti import AFIETI
    prob = W.config("C3")
    s = Solver(prob, prec="tf32", tol=1e-8, use_graph=True, maxit=4000)
    try:
        off = prob.offsets()
        rng = np.random.default_rng(8)
        x = W.torn_random(prob, 51)[0]
        y = s.apply(A.AFI_OP_STIFFNESS, torch.from_numpy(x).cuda()).cpu().numpy()
        for _ in range(6):
            k = int(rng.integers(prob.npatch))
            im = [int(rng.integers(n)) for n in prob.n(k)]
            Ax, _, _, N = node_rows(prob, k, im, x[off[k]:off[k + 1]])
            node = im[0] + prob.n(k)[0] * (im[1] + prob.n(k)[1] * im[2])
            got = np.array([y[off[k] + l * N + node] for l in range(3)])
            np.testing.assert_allclose(got, Ax, rtol=1e-11, atol=1e-11 * np.abs(Ax).max())
        r = W.torn_random(prob, 52)[0]
        sizes = [int(np.prod(prob.n(k))) for k in range(prob.npatch)]
        big, small = int(np.argmax(sizes)), int(np.argmin(sizes))
        for prec, tol in (("fp64", 1e-10), ("tf32", 1e-2)):
            s.set_precision(prec)
            out = s.fd(torch.from_numpy(r).cuda()).cpu().numpy()
            for k in (big, small):
                N = sizes[k]
                for l in (0, 2):
                    a = off[k] + l * N
                    ref = fd_block_ref(prob, k, l, r[a:a + N])
                    err = np.linalg.norm(out[a:a + N] - ref) / np.linalg.norm(ref)
                    assert err < tol, (prec, k, l, err)
        s.set_precision("tf32")
        f = s.load_vector(W.body_force_coeffs(prob))
        u, lam = s.solve(f)
        assert s.last_info["relres_true"] <= 1e-8
        orc = AFIETI(prob)
        un, ln, fn = u.cpu().numpy(), lam.cpu().numpy(), f.cpu().numpy()
        assert np.linalg.norm(orc.B @ un) <= 1e-7 * np.linalg.norm(un)
        btl = orc.B.T @ ln
        scale = np.abs(fn).max()
        for _ in range(5):
            k = int(rng.integers(prob.npatch))
            im = [int(rng.integers(n)) for n in prob.n(k)]
            im[int(rng.integers(3))] = 0
            Au, _, _, N = node_rows(prob, k, im, un[off[k]:off[k + 1]])
            node = im[0] + prob.n(k)[0] * (im[1] + prob.n(k)[1] * im[2])
            for l in range(3):
                i = off[k] + l * N + node
                assert abs(fn[i] - Au[l] - btl[i]) <= 1e-6 * scale
    finally:
        s.close()


def test_c5_local_only_fd_two_rhs():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    from paper_2001_09626_gb300 import afieti as A
    prob = W.config("C5")
    s = Solver(prob, prec="tf32", local_only=True)
    try:
        with pytest.raises(A.AfiError):
            s.solve(torch.zeros(s.n_dof, dtype=torch.float64, device="cuda"))
        r = torch.from_numpy(W.torn_random(prob, 61, nrhs=2)).cuda()
        off = prob.offsets()
        N = int(np.prod(prob.n(0)))
        for prec, tol in (("fp64", 1e-10), ("tf32", 1e-2), ("bf16", 3e-2)):
            s.set_precision(prec)
            out = s.fd(r)
            for j, k, l in ((0, 0, 0), (1, 137, 2), (1, 255, 1)):
                a = int(off[k]) + l * N
                rb = r[j, a:a + N].cpu().numpy()
                ref = fd_block_ref(prob, k, l, rb)
                err = np.linalg.norm(out[j, a:a + N].cpu().numpy() - ref) / np.linalg.norm(ref)
                assert err < tol, (prec, j, k, l, err)
    finally:
        s.close()
