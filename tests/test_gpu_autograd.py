"""The torch.autograd.Function IetiSolve: u = IetiSolve.apply(f, lame, solver),
then .backward() on the compliance J = f^T u.

Autograd forms dJ/df = u + z, with z the adjoint state solving the same
saddle system for the right-hand side dJ/du = f (so z = u), and dJ/dlame
from afi_lame_grad(u, z) = -z^T (dA/dtheta) u.  The oracle's
compliance_and_grads gives (J, 2u, -u^T A_lam^(k) u, -u^T A_mu^(k) u) from
its conforming direct solve.  Both gradients are compared at 1e-7 relative
(FP64 solves at tolerance 1e-10)."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import adjoint
from oracle.ieti import AFIETI

from blocks import block_rel, torn_blocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,prec", [("C1-small", "fp64"), ("C2-small", "fp64"),
                                       ("C4-small", "tf32")])
def test_ietisolve_backward_matches_oracle_adjoint(name, prec):
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import IetiSolve, Solver
    prob = W.config(name)
    orc = AFIETI(prob)
    fo = orc.load(W.body_force_coeffs(prob))
    J_ref, dJdf_ref, dJdlame_ref = adjoint.compliance_and_grads(orc, fo)
    s = Solver(prob, prec=prec, tol=1e-10)
    try:
        f = torch.from_numpy(fo.copy()).cuda().requires_grad_(True)
        lame = torch.from_numpy(prob.lame.copy()).cuda().requires_grad_(True)
        u = IetiSolve.apply(f, lame, s)
        J = torch.dot(f, u)
        J.backward()
        torch.cuda.synchronize()
        assert abs(float(J.detach()) - J_ref) <= 1e-9 * abs(J_ref)
        assert block_rel(f.grad.cpu().numpy(), dJdf_ref, torn_blocks(orc)) < 1e-7
        gl = lame.grad.cpu().numpy()
        assert gl.shape == dJdlame_ref.shape
        assert np.all(np.abs(gl - dJdlame_ref) <= 1e-7 * np.abs(dJdlame_ref)
                      + 1e-9 * np.abs(dJdlame_ref).max()), (gl, dJdlame_ref)
    finally:
        s.close()


def test_ietisolve_gradient_of_a_linear_functional():
    """J = g^T u for a fixed random g: dJ/df = z solves the adjoint system, so
    f.grad must equal the oracle's direct solve for the right-hand side g
    (the u part of the saddle solution), and the Lame gradient is
    -z^T (dA/dtheta) u."""
    import __graft_entry__ as gb
    gb.build()
    from paper_2001_09626_gb300.solver import IetiSolve, Solver
    prob = W.config("C2-small")
    orc = AFIETI(prob)
    fo = orc.load(W.body_force_coeffs(prob))
    gvec = W.torn_random(prob, 77)[0]
    u_ref, _ = orc.direct_solve(fo)
    z_ref, _ = orc.direct_solve(gvec)
    lame_ref = adjoint.lame_gradient(orc, u_ref, z_ref)
    s = Solver(prob, prec="fp64", tol=1e-10)
    try:
        f = torch.from_numpy(fo.copy()).cuda().requires_grad_(True)
        lame = torch.from_numpy(prob.lame.copy()).cuda().requires_grad_(True)
        u = IetiSolve.apply(f, lame, s)
        (torch.from_numpy(gvec).cuda() * u).sum().backward()
        assert block_rel(f.grad.cpu().numpy(), z_ref, torn_blocks(orc)) < 1e-7
        gl = lame.grad.cpu().numpy()
        assert np.all(np.abs(gl - lame_ref) <= 1e-7 * np.abs(lame_ref)
                      + 1e-9 * np.abs(lame_ref).max()), (gl, lame_ref)
    finally:
        s.close()
