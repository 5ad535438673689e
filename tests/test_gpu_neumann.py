"""GPU parity with natural (zero-traction) outer faces: the x-faces of the
jittered cube (C2-small) and of the 2D square (C1) are free, the other outer
faces Dirichlet.  Patches away from the Dirichlet faces float; the AF-IETI
solve through the C ABI must still give the conforming Galerkin solution."""
import numpy as np
import pytest

import afi_workloads as W
from oracle.ieti import AFIETI

from blocks import block_rel, mult_blocks, saddle_blocks, torn_blocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["C2-small", "C1"])
def neumann(request):
    import __graft_entry__ as g
    g.build()
    prob = W.with_neumann(W.config(request.param), (0, 1))
    orc = AFIETI(prob)
    f = orc.load(W.body_force_coeffs(prob))
    ud, _ = orc.direct_solve(f)
    _, _, info = orc.solve(f, tol=1e-10)
    return prob, orc, f, ud, info["iters"]


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
def test_neumann_solve_matches_direct(neumann, prec):
    from paper_2001_09626_gb300.solver import Solver
    prob, orc, f, ud, it_oracle = neumann
    s = Solver(prob, prec=prec, tol=1e-10, use_graph=True)
    try:
        assert s.n_c == orc.nc
        u, _ = s.solve(torch.from_numpy(f).cuda())
        u = u.cpu().numpy()
        assert block_rel(u, ud, torn_blocks(orc)) <= 1e-7
        assert s.last_info["relres_true"] <= 1e-10
        if prec == "fp64":
            assert abs(s.last_info["iters"] - it_oracle) <= max(2, 0.05 * it_oracle)
    finally:
        s.close()


def test_neumann_PS_and_preconditioner(neumann):
    """Shell dofs on a free face that lie on no interface have no constraint
    row, so B^T leaves them zero; P_S and the preconditioner must match the
    oracle there too."""
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    prob, orc, _, _, _ = neumann
    s = Solver(prob, prec="fp64", tol=1e-10)
    try:
        rng = np.random.default_rng(21)
        T = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
        lam = rng.uniform(-1, 1, orc.nc)
        ps = s.apply(A.AFI_OP_PS, T(lam)).cpu().numpy()
        ref = orc.P_S(lam)
        assert block_rel(ps, ref, mult_blocks(orc)) <= 1e-10
        x = rng.uniform(-1, 1, orc.ndof + orc.nc)
        z = s.apply(A.AFI_OP_PRECOND, T(x)).cpu().numpy()
        refz = np.concatenate(orc.precond_apply(x[:orc.ndof], x[orc.ndof:]))
        assert block_rel(z, refz, saddle_blocks(orc)) <= 1e-10
    finally:
        s.close()
