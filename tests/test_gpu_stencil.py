"""The two stiffness forms (eqs. 3.1, 4.2) against the oracle: the
iterations' double-FP32 form (a row-compressed copy of the stencil with each
coefficient and input held as a sum of two FP32 numbers, products summed with
exact product errors and TwoSum) and the FP64 stencil, which the true residual
and AFI_VARIANT_STENCIL_F64 use.

Element-wise bound for the double-FP32 form, with u = 2^-24 and N the number
of products in a row: splitting a and x costs at most u^2 (|a| |x|) each, the
dropped lo*lo term and the rounding of the cross terms 3 u^2 |a x|, and the
FP32 sum of the N addition errors at most N u^2 max |partial sum|; so
|y - A x| <= (N + 8) u^2 (|A| |x|) covers it, with the oracle's FP64 error
(N 2^-53 (|A| |x|)) far below."""
import numpy as np
import pytest

import afi_workloads as W
from oracle.ieti import AFIETI

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# configurations, plus uneven patches of degree 5 and 2 (rows of several
# lengths per tile, the largest neighbour stencil)
MAKERS = {
    "C1": lambda: W.config("C1"),
    "C2-small": lambda: W.config("C2-small"),
    "C5-small": lambda: W.config("C5-small"),
    "annulus-p5-uneven": lambda: W.quarter_annulus(grid=(2, 1, 1), p=5, nel_cols=[[3, 5], [4], [3]],
                                                   name="annulus-p5-uneven"),
    "annulus-p2-uneven": lambda: W.quarter_annulus(grid=(2, 1, 2), p=2, nel_cols=[[6, 3], [5], [2, 7]],
                                                   name="annulus-p2-uneven"),
}
CASES = list(MAKERS)


def nprod(prob):
    """Products the kernels form per row: d (2p+1)^d."""
    p = int(max(prob.degree))
    return prob.dim * (2 * p + 1) ** prob.dim


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.fixture(scope="module", params=CASES)
def pair(request):
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = MAKERS[request.param]()
    orc = AFIETI(prob)
    orc.assemble()
    sd = Solver(prob, prec="fp64", tol=1e-10)
    s64 = Solver(prob, prec="fp64", tol=1e-10, stencil_f64=True)
    yield request.param, prob, orc, sd, s64
    sd.close()
    s64.close()


def test_elementwise_bound(pair):
    from paper_2001_09626_gb300 import afieti as A
    _, prob, orc, sd, s64 = pair
    absA = abs(orc.A)
    nrow = nprod(prob)
    u2 = 2.0 ** -48
    for seed in (11, 12):
        x = W.torn_random(prob, seed)[0]
        ref = orc.A @ x
        mag = absA @ np.abs(x)
        yd = sd.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        y64 = s64.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
        assert np.all(np.abs(yd - ref) <= (nrow + 8) * u2 * mag + 1e-300)
        assert np.all(np.abs(y64 - ref) <= 2 * nrow * 2.0 ** -53 * mag + 1e-300)
        assert np.linalg.norm(yd - ref) <= 1e-11 * np.linalg.norm(ref)


def test_rigid_modes_and_scaling(pair):
    """A R = 0 holds to the rounding level of |A| |R|, and scaling x by a
    power of two scales y exactly (both splits are exact under it)."""
    from paper_2001_09626_gb300 import afieti as A
    _, prob, orc, sd, _ = pair
    Rd = orc.R.toarray()
    absA = abs(orc.A)
    nrow = nprod(prob)
    for j in (0, Rd.shape[1] - 1):
        y = sd.apply(A.AFI_OP_STIFFNESS, T(Rd[:, j])).cpu().numpy()
        assert np.all(np.abs(y) <= (nrow + 8) * 2.0 ** -48 * (absA @ np.abs(Rd[:, j])) + 1e-300)
    x = W.torn_random(prob, 13)[0]
    y1 = sd.apply(A.AFI_OP_STIFFNESS, T(x)).cpu().numpy()
    y2 = sd.apply(A.AFI_OP_STIFFNESS, T(x * 2.0 ** -20)).cpu().numpy()
    np.testing.assert_array_equal(y2, y1 * 2.0 ** -20)


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_solves_agree(pair, prec):
    name, prob, orc, sd, s64 = pair
    f = orc.load(W.body_force_coeffs(prob))
    ud, _ = orc.direct_solve(f)
    its = []
    for s in (sd, s64):
        s.set_precision(prec)
        try:
            u, _ = s.solve(T(f))
            assert s.last_info["relres_true"] <= 1e-10
            assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-7 * np.linalg.norm(ud)
            its.append(s.last_info["iters"])
            assert s.last_info["fp64_restarts"] == 0
        finally:
            s.set_precision("fp64")
    # the forms differ by rounding only: the stopping iteration may move by a
    # period of the true-residual check schedule (5 or more iterations)
    assert abs(its[0] - its[1]) <= max(5, 0.03 * max(its)), its


def test_memory_of_the_pair_copy(pair):
    from paper_2001_09626_gb300 import afieti as A
    _, _, _, sd, s64 = pair
    assert A.afi_memory(sd.ctx)[1] == 2 * A.afi_memory(s64.ctx)[1]


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_fp64_restart(pair, prec):
    """The restart a stalled double-FP32 iteration takes (forced here at the
    first true-residual check): MINRES continues from the iterate with the
    FP64 stiffness on b - calA x0 and returns x0 + d, the same solution."""
    from paper_2001_09626_gb300.solver import Solver
    name, prob, orc, sd, _ = pair
    f = orc.load(W.body_force_coeffs(prob))
    ud, ld = orc.direct_solve(f)
    sr = Solver(prob, prec=prec, tol=1e-10, force_restart=True)
    try:
        u, lam = sr.solve(T(f))
        info = sr.last_info
        assert info["fp64_restarts"] == 1
        assert info["relres_true"] <= 1e-10
        assert np.linalg.norm(u.cpu().numpy() - ud) <= 1e-7 * np.linalg.norm(ud)
        assert np.linalg.norm(lam.cpu().numpy() - ld) <= 1e-7 * np.linalg.norm(ld)
    finally:
        sr.close()
