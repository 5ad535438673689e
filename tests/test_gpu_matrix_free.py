"""The matrix-free stiffness and mass (AFI_VARIANT_MATRIX_FREE, eqs. 3.1 and
4.8 by sum factorisation over each element) against the oracle's assembled
quadrature sums, through the C ABI.

Tolerances.  Both sides integrate with the same Gauss rule, so they differ
by rounding only.
  * FP64 form: every product the kernel forms is a sum over the (p+1)^3
    Gauss points of one element of terms of size at most those of the
    assembled entries; the errors stay below n_ops 2^-53 times the terms'
    magnitudes.  With a few hundred operations per entry and the entries'
    internal cancellation, 1e-11 (|A| |x|)_i bounds it.
  * FP32 form: the same with 2^-24 (6e-8): 2e-4 (|A| |x|)_i, and 1e-5 of the
    norm for a random input.
  * Solves: the mixed form (TF32 local solvers, FP32 products refined against
    the FP64 true residual) must meet the FP64 tolerance 1e-8 on the true
    residual and a solution error of 1e-6; the FP64 form, 1e-10 and
    1e-7 (the tolerances of the stored-stencil solves).
The full-size rows are C5-mid's (the C5 patch: p = 4, 48^3 elements), from
the oracle's quadrature over each sampled node's support."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import assembly
from oracle.ieti import AFIETI

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAKERS = {
    "C2-small": lambda: W.config("C2-small"),
    "C5-small": lambda: W.config("C5-small"),
    "annulus-p2-uneven": lambda: W.quarter_annulus(grid=(2, 1, 2), p=2, nel_cols=[[6, 3], [5], [2, 7]],
                                                   name="annulus-p2-uneven"),
    "annulus-p5-uneven": lambda: W.quarter_annulus(grid=(2, 1, 1), p=5, nel_cols=[[3, 5], [4], [3]],
                                                   name="annulus-p5-uneven"),
}
CASES = list(MAKERS)


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.fixture(scope="module", params=CASES)
def ctxs(request):
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = MAKERS[request.param]()
    orc = AFIETI(prob)
    orc.assemble()
    s32 = Solver(prob, prec="tf32", tol=1e-8, matrix_free=True)
    s64 = Solver(prob, prec="fp64", tol=1e-10, matrix_free=True, stencil_f64=True)
    yield request.param, prob, orc, s32, s64
    s32.close()
    s64.close()


def test_stiffness_elementwise(ctxs):
    from paper_2001_09626_gb300 import afieti as A
    _, prob, orc, s32, s64 = ctxs
    absA = abs(orc.A)
    for seed in (21, 22):
        x = W.torn_random(prob, seed)[0]
        ref = orc.A @ x
        mag = absA @ np.abs(x)
        y64 = s64.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        y32 = s32.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        assert np.all(np.abs(y64 - ref) <= 1e-11 * mag + 1e-300)
        assert np.all(np.abs(y32 - ref) <= 2e-4 * mag + 1e-300)
        assert np.linalg.norm(y32 - ref) <= 1e-5 * np.linalg.norm(ref)
        assert np.linalg.norm(y64 - ref) <= 1e-13 * np.linalg.norm(ref)


def test_rigid_modes_in_the_kernel(ctxs):
    """A R = 0 (the rigid motions lie in the spline space, Section 4) to the
    rounding level of |A| |R|."""
    from paper_2001_09626_gb300 import afieti as A
    _, prob, orc, s32, s64 = ctxs
    Rd = orc.R.toarray()
    absA = abs(orc.A)
    for j in range(Rd.shape[1]):
        mag = absA @ np.abs(Rd[:, j])
        y = s64.apply(A.AFI_OP_STIFFNESS, T(Rd[:, j])).cpu().numpy()
        assert np.all(np.abs(y) <= 1e-11 * mag + 1e-300)


def test_load_vector(ctxs):
    """f = M c with the mapped mass (eq. 4.8), matrix-free against the oracle."""
    _, prob, orc, s32, s64 = ctxs
    coeffs = W.body_force_coeffs(prob)
    fo = orc.load(coeffs)
    for s in (s32, s64):
        f = s.load_vector(coeffs).cpu().numpy()
        np.testing.assert_allclose(f, fo, rtol=1e-12, atol=1e-14 * np.abs(fo).max())


def test_solves(ctxs):
    name, prob, orc, s32, s64 = ctxs
    f = orc.load(W.body_force_coeffs(prob))
    ud, ld = orc.direct_solve(f)
    u, lam = s32.solve(T(f))
    info = s32.last_info
    assert info["relres_true"] <= 1e-8, info
    assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-6 * np.linalg.norm(ud)
    assert np.linalg.norm(lam.cpu().numpy() - ld) <= 1e-6 * np.linalg.norm(ld)
    it_mixed = info["iters"]
    u, lam = s64.solve(T(f))
    info = s64.last_info
    assert info["relres_true"] <= 1e-10, info
    assert info["fp64_restarts"] == 0
    assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-7 * np.linalg.norm(ud)
    assert np.linalg.norm(lam.cpu().numpy() - ld) <= 1e-7 * np.linalg.norm(ld)
    # the same FP64 method as the oracle's AF-IETI: iteration counts within
    # the true-residual check period
    ro = orc.solve(f, tol=1e-10)[2]["iters"]
    assert abs(info["iters"] - ro) <= max(5, 0.05 * ro), (info["iters"], ro)
    # the refined FP32 products cost few extra iterations over the FP64 ones
    assert it_mixed <= 1.6 * info["iters"] + 20, (it_mixed, info["iters"])


def test_matches_the_stored_stencil(ctxs):
    """Same operator as the assembled FP64 stencil, to rounding."""
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    _, prob, orc, _, s64 = ctxs
    sd = Solver(prob, prec="fp64", tol=1e-10, stencil_f64=True)
    try:
        x = W.torn_random(prob, 23)[0]
        ys = sd.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        ym = s64.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        mag = abs(orc.A) @ np.abs(x)
        assert np.all(np.abs(ys - ym) <= 1e-11 * mag + 1e-300)
        assert A.afi_memory(s64.ctx)[1] == 0
    finally:
        sd.close()


def node_rows(prob, k, i_multi, x_patch):
    g = assembly.PatchGeometry(prob.ctrl[k], prob.degree[k], prob.nel[k])
    lam, mu = prob.lame[k]
    qr, cr = g.support_q(i_multi), g.neighbour_c(i_multi)
    A, cols = assembly.stiffness_block(g, lam, mu, qr, cr)
    Mm, _ = assembly.mass_block(g, qr, cr)
    node = sum(i_multi[l] * int(np.prod(g.ns[:l])) for l in range(g.dim))
    loc = int(np.where(cols == node)[0][0])
    nc = len(cols)
    N = int(np.prod(g.ns))
    xs = np.concatenate([x_patch[l * N + cols] for l in range(3)])
    Ax = np.array([A[l * nc + loc] @ xs for l in range(3)])
    magr = np.array([np.abs(A[l * nc + loc]) @ np.abs(xs) for l in range(3)])
    return Ax, magr, Mm[loc], cols, N


def test_c5_patch_sampled_rows():
    """C5's patch shape (p = 4, 48^3 elements, twisted box) at full size:
    sampled rows of A x and M c against the oracle's quadrature over each
    node's support, the FP64 and FP32 products."""
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config("C5-mid")
    s64 = Solver(prob, prec="tf32", tol=1e-8, matrix_free=True, stencil_f64=True)
    s32 = Solver(prob, prec="tf32", tol=1e-8, matrix_free=True)
    try:
        rng = np.random.default_rng(7)
        coeffs = W.body_force_coeffs(prob)
        f = s64.load_vector(coeffs).cpu().numpy()
        x = W.torn_random(prob, 41)[0]
        y64 = s64.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        y32 = s32.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        off = prob.offsets()
        for it in range(10):
            k = int(rng.integers(prob.npatch))
            im = [int(rng.integers(n)) for n in prob.n(k)]
            if it < 3:   # faces, edges and corners of the patch
                im = [0 if rng.random() < 0.5 else n - 1 for n in prob.n(k)]
            Ax, magr, mrow, cols, N = node_rows(prob, k, im, x[off[k]:off[k + 1]])
            node = im[0] + prob.n(k)[0] * (im[1] + prob.n(k)[1] * im[2])
            got64 = np.array([y64[off[k] + l * N + node] for l in range(3)])
            got32 = np.array([y32[off[k] + l * N + node] for l in range(3)])
            assert np.all(np.abs(got64 - Ax) <= 1e-11 * magr), (got64, Ax)
            assert np.all(np.abs(got32 - Ax) <= 2e-4 * magr), (got32, Ax)
            cf = coeffs[k].reshape(3, -1)
            ref_f = np.array([mrow @ cf[l][cols] for l in range(3)])
            got_f = np.array([f[off[k] + l * N + node] for l in range(3)])
            np.testing.assert_allclose(got_f, ref_f, rtol=1e-12, atol=1e-15)
    finally:
        s64.close()
        s32.close()
