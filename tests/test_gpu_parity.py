"""GPU parity of every hot-path operator against the CPU oracle, through the
C ABI, on seeded inputs spanning several tiles and ragged sizes (2D and 3D,
degrees 2-4, identity, jittered, annulus and twisted geometries).

Tolerances (FP64 paths): operators that are sums of O(10^3) products are
compared at 1e-11 relative to the norm of the result; solves at 1e-7
relative (tolerance 1e-10 of the iterative solve against the direct solve).
FP32 local solvers: 2e-5 relative per application (FP32 unit roundoff times
the O(n) accumulation length and the conditioning of U); TF32 (operands
truncated to a 10-bit mantissa, error up to 9.8e-4 each) 1e-2 and BF16 (7-bit
mantissa, 3.9e-3) 3e-2 per application, the same accumulation argument over
six mode products.  Whatever the local-solver
precision, the converged solution is compared at 1e-7 (the preconditioner
changes only the iteration)."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import fd as ofd
from oracle.ieti import AFIETI

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = ["C1-small", "C1", "C2-small", "C4-small", "C5-small"]


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module", params=CASES)
def case(request):
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config(request.param)
    orc = AFIETI(prob)
    orc.assemble()
    s = Solver(prob, prec="fp64", tol=1e-10)
    yield request.param, prob, orc, s
    s.close()


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def test_sizes(case):
    _, _, orc, s = case
    assert (s.n_dof, s.n_c) == (orc.ndof, orc.nc)


def test_load_vector(case):
    _, prob, orc, s = case
    c = W.body_force_coeffs(prob)
    f = s.load_vector(c).cpu().numpy()
    assert rel(f, orc.load(c)) < 1e-13


def test_stiffness_matvec(case):
    _, prob, orc, s = case
    from paper_2001_09626_gb300 import afieti as A
    x = W.torn_random(prob, 11)[0]
    y = s.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
    assert rel(y, orc.A @ x) < 1e-11


def test_jumps_and_projections(case):
    _, prob, orc, s = case
    from paper_2001_09626_gb300 import afieti as A
    x = W.torn_random(prob, 12)[0]
    lam = np.random.default_rng(3).uniform(-1, 1, orc.nc)
    np.testing.assert_array_equal(s.apply(A.AFI_OP_B, T(x)).cpu().numpy(), orc.B @ x)
    np.testing.assert_allclose(s.apply(A.AFI_OP_BT, T(lam)).cpu().numpy(), orc.B.T @ lam,
                               rtol=0, atol=1e-15)
    assert rel(s.apply(A.AFI_OP_PCHI, T(lam)).cpu().numpy(), orc.P_chi(lam)) < 1e-10
    assert rel(s.apply(A.AFI_OP_PU, T(x)).cpu().numpy(), orc.P_u(x)) < 1e-11


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5), ("tf32", 1e-2),
                                      ("bf16", 3e-2)])
def test_fd_apply(case, prec, tol):
    _, prob, orc, s = case
    from paper_2001_09626_gb300 import afieti as A
    s.set_precision(prec)
    try:
        x = W.torn_random(prob, 13)[0]
        y = s.apply(A.AFI_OP_PA_INV, T(x)).cpu().numpy()
        assert rel(y, orc.PA_inv(x)) < tol
    finally:
        s.set_precision("fp64")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5), ("tf32", 1e-2),
                                      ("bf16", 3e-2)])
def test_interior_fd(case, prec, tol):
    _, prob, orc, s = case
    s.set_precision(prec)
    try:
        loc = orc._local()
        blocks, refs = [], []
        rng = np.random.default_rng(14)
        for k, (per, mask, Hs) in enumerate(loc):
            for l in range(orc.dim):
                r = rng.uniform(-1, 1, int(mask.sum()))
                blocks.append(r)
                refs.append(per[l][2].solve(r))
        r = np.concatenate(blocks)
        out = s.fd(T(r), interior=True).cpu().numpy()
        assert rel(out, np.concatenate(refs)) < tol
    finally:
        s.set_precision("fp64")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_schur_and_PS(case, prec, tol):
    _, prob, orc, s = case
    from paper_2001_09626_gb300 import afieti as A
    s.set_precision(prec)
    try:
        t = W.torn_random(prob, 15)[0] * orc.shell
        y = s.apply(A.AFI_OP_SCHUR, T(t)).cpu().numpy()
        assert rel(y, orc.S_hat_H(t)) < tol
        lam = np.random.default_rng(4).uniform(-1, 1, orc.nc)
        assert rel(s.apply(A.AFI_OP_PS, T(lam)).cpu().numpy(), orc.P_S(lam)) < tol
    finally:
        s.set_precision("fp64")


def test_precond_and_saddle(case):
    _, prob, orc, s = case
    from paper_2001_09626_gb300 import afieti as A
    rng = np.random.default_rng(16)
    x = rng.uniform(-1, 1, orc.ndof + orc.nc)
    y = s.apply(A.AFI_OP_SADDLE, T(x)).cpu().numpy()
    ref = np.concatenate(orc.op(x[:orc.ndof], x[orc.ndof:]))
    assert rel(y, ref) < 1e-11
    z = s.apply(A.AFI_OP_PRECOND, T(x)).cpu().numpy()
    refz = np.concatenate(orc.precond_apply(x[:orc.ndof], x[orc.ndof:]))
    assert rel(z, refz) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_solve_matches_direct(case, prec):
    name, prob, orc, s = case
    s.set_precision(prec)
    try:
        c = W.body_force_coeffs(prob)
        f = orc.load(c)
        u, lam = s.solve(T(f))
        info = s.last_info
        ud, ld = orc.direct_solve(f)
        assert info["relres_true"] <= 1e-10
        assert rel(u.cpu().numpy(), ud) < 1e-7
        assert rel(lam.cpu().numpy(), ld) < 1e-7
        assert np.linalg.norm(orc.B @ u.cpu().numpy()) < 1e-8 * np.linalg.norm(ud)
        if prec == "fp64":
            # same iterates; the stopping iteration follows the true-residual
            # check schedule, which rounding can move by a few iterations
            _, _, oinfo = orc.solve(f, tol=1e-10)
            assert abs(info["iters"] - oinfo["iters"]) <= max(2, 0.05 * oinfo["iters"]), \
                (info["iters"], oinfo["iters"])
    finally:
        s.set_precision("fp64")


def test_adjoint_gradients(case):
    name, prob, orc, s = case
    from oracle import adjoint
    f = orc.load(W.body_force_coeffs(prob))
    u, _ = s.solve(T(f))
    g = s.lame_grad(u, u).cpu().numpy()
    ud, _ = orc.direct_solve(f)
    ref = adjoint.lame_gradient(orc, ud, ud)
    assert rel(g, ref) < 1e-7
    # adjoint state for J = f^T u equals u
    z2, _ = s.solve_adjoint(T(f))
    assert rel(z2.cpu().numpy(), ud) < 1e-7


def test_invalid_arguments(case):
    _, prob, orc, s = case
    from paper_2001_09626_gb300 import afieti as A
    x = T(np.zeros(orc.ndof))
    with pytest.raises(A.AfiError):
        A.fd_apply(s.ctx, 2, x, x, 1)
    with pytest.raises(A.AfiError):
        A.fd_apply(s.ctx, 0, x, x, 0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_replay_matches_eager(case, prec):
    """Six captured iterations replayed as a CUDA graph give the same iterates
    (bitwise) and iteration count as launching every kernel from the host."""
    name, prob, orc, s = case
    from paper_2001_09626_gb300.solver import Solver
    f = T(orc.load(W.body_force_coeffs(prob)))
    s.set_precision(prec)
    try:
        u0, l0 = s.solve(f)
        it0 = s.last_info["iters"]
        g = Solver(prob, prec=prec, tol=1e-10, use_graph=True)
        try:
            u1, l1 = g.solve(f)
            assert g.last_info["iters"] == it0
            assert torch.equal(u0, u1) and torch.equal(l0, l1)
            u2, _ = g.solve(f)            # replaying the cached graph again
            assert torch.equal(u1, u2)
        finally:
            g.close()
    finally:
        s.set_precision("fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_fd_batched_rhs(case, prec):
    """fd_apply on a batch of right-hand sides (one launch) equals the
    applications one by one."""
    _, prob, orc, s = case
    s.set_precision(prec)
    try:
        R = T(W.torn_random(prob, 41, nrhs=3))
        batch = s.fd(R)
        for j in range(3):
            assert torch.equal(batch[j], s.fd(R[j].contiguous()))
        Ri = T(np.random.default_rng(2).uniform(-1, 1, (2, sum(int(m.sum()) * orc.dim
                                                             for _, m, _ in orc._local()))))
        bi = s.fd(Ri, interior=True)
        for j in range(2):
            assert torch.equal(bi[j], s.fd(Ri[j].contiguous(), interior=True))
    finally:
        s.set_precision("fp64")


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_fd_special_values(case, prec):
    """The mixed-precision FD converts FP64 <-> FP32 with integer bit
    operations: zero maps to zero, scaling the input by a power of two
    scales the output by the same power exactly (exponent handling), and a
    NaN spreads over its own (patch, component) block only."""
    _, prob, orc, s = case
    s.set_precision(prec)
    try:
        x = W.torn_random(prob, 17)[0]
        z = s.fd(T(np.zeros_like(x))).cpu().numpy()
        assert np.all(z == 0.0)
        y = s.fd(T(x)).cpu().numpy()
        for e in (-20, 20):
            ys = s.fd(T(np.ldexp(x, e))).cpu().numpy()
            assert np.array_equal(ys, np.ldexp(y, e))
        k = prob.npatch // 2
        lo = int(orc.off[k]) + orc.N[k]          # component 1 of patch k
        hi = lo + orc.N[k]
        xn = x.copy()
        xn[lo + orc.N[k] // 3] = np.nan
        yn = s.fd(T(xn)).cpu().numpy()
        assert np.all(np.isnan(yn[lo:hi]))
        assert np.array_equal(yn[:lo], y[:lo]) and np.array_equal(yn[hi:], y[hi:])
    finally:
        s.set_precision("fp64")
