"""EXACT local solvers (Section 5.1) on the GPU against the oracle's:
P_A^ex = A + D_H M applied through dense per-patch inverses, the exact
Schur complements S^(k) and P_S^{ex-nr} (Remark 1), the preconditioner, and
the solve, whose iteration count is the paper's reference for the inexact
solvers (EXACT needs fewer iterations).  Tolerances: the dense FP64 inverses
lose about the condition number of the local matrices (<= 1e4 here), so the
operators are compared at 1e-10 relative and the solves at 1e-7."""
import numpy as np
import pytest

import afi_workloads as W
from oracle.ieti import AFIETI

from blocks import block_rel, mult_blocks, saddle_blocks, torn_blocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = ["C1", "C4-small"]


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.fixture(scope="module", params=CASES)
def case(request):
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config(request.param)
    orc = AFIETI(prob, precond="exact")
    orc.assemble()
    s = Solver(prob, prec="fp64", tol=1e-10, exact=True)
    yield request.param, prob, orc, s
    s.close()


def test_exact_operators(case):
    from paper_2001_09626_gb300 import afieti as A
    _, prob, orc, s = case
    x = W.torn_random(prob, 21)[0]
    assert block_rel(s.apply(A.AFI_OP_PA_INV, T(x)).cpu().numpy(), orc.PA_inv_exact(x),
                     torn_blocks(orc)) < 1e-10
    t = W.torn_random(prob, 22)[0] * orc.shell
    assert block_rel(s.apply(A.AFI_OP_SCHUR, T(t)).cpu().numpy(), orc.S_exact(t),
                     torn_blocks(orc)) < 1e-10
    lam = np.random.default_rng(23).uniform(-1, 1, orc.nc)
    assert block_rel(s.apply(A.AFI_OP_PS, T(lam)).cpu().numpy(), orc.P_S_exact(lam),
                     mult_blocks(orc)) < 1e-10
    z = np.random.default_rng(24).uniform(-1, 1, orc.ndof + orc.nc)
    ref = np.concatenate(orc.precond_apply(z[:orc.ndof], z[orc.ndof:]))
    assert block_rel(s.apply(A.AFI_OP_PRECOND, T(z)).cpu().numpy(), ref, saddle_blocks(orc)) < 1e-10


def test_exact_schur_kills_rigid_traces(case):
    """A R = 0, so the harmonic extension of a rigid mode's shell trace is the
    mode itself and S maps the trace to zero."""
    from paper_2001_09626_gb300 import afieti as A
    _, prob, orc, s = case
    Rd = orc.R.toarray()
    for j in (0, Rd.shape[1] - 1):
        t = Rd[:, j] * orc.shell
        y = s.apply(A.AFI_OP_SCHUR, T(t)).cpu().numpy()
        assert np.linalg.norm(y) <= 1e-10 * np.linalg.norm(t)


def test_exact_solve(case):
    from paper_2001_09626_gb300.solver import Solver
    name, prob, orc, s = case
    f = orc.load(W.body_force_coeffs(prob))
    u, lam = s.solve(T(f))
    info = s.last_info
    ud, ld = orc.direct_solve(f)
    assert info["relres_true"] <= 1e-10
    assert block_rel(u.cpu().numpy(), ud, torn_blocks(orc)) < 1e-7
    assert block_rel(lam.cpu().numpy(), ld, mult_blocks(orc)) < 1e-7
    _, _, oinfo = orc.solve(f, tol=1e-10)
    assert abs(info["iters"] - oinfo["iters"]) <= max(2, 0.05 * oinfo["iters"]), (info["iters"], oinfo["iters"])
    si = Solver(prob, prec="fp64", tol=1e-10)
    try:
        si.solve(T(f))
        assert info["iters"] < si.last_info["iters"]   # EXACT < INEXACT, as in the paper's tables
    finally:
        si.close()


def test_exact_rejects_large_patches():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    prob = W.unit_box(3, (1, 1, 1), 3, 13, name="box-n16")   # 3 * 16^3 = 12288 dofs
    with pytest.raises(A.AfiError):
        Solver(prob, prec="fp64", exact=True)
    assert "4096" in A.afi_last_error()
