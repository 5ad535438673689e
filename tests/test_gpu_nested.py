"""Nested non-conforming interfaces on the GPU (Section 2; the paper's
non-conforming test of Section 6: a box of three patches with 4, 8 and 16
elements per direction).  The operator-level parity of these problems is in
test_gpu_parity.py (cases NC-small, NC3-small); here:

- the knot-insertion rows found by the library equal the oracle's (whose
  weights come from an L2 projection, not from knot insertion);
- the GPU solve reproduces a quadratic displacement that vanishes on the
  boundary exactly (it lies in the constrained space, and the quadrature is
  exact for it), at FP64 and TF32 local solvers, on the oracle-sized boxes
  and on the paper's 4/8/16 box;
- a nested face with an edge off the Dirichlet boundary is refused.
"""
import dataclasses

import numpy as np
import pytest

import afi_workloads as W
from oracle.ieti import AFIETI

from test_oracle_nested import CASES as POLY_CASES, polynomial_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    return A, Solver


@pytest.mark.parametrize("name", ["NC-small", "NC3-small"])
def test_nested_rows_equal_the_oracle(lib, name):
    """B and B^T on unit vectors of every nested dof: the same rows, the same
    weights (to rounding), in the same order."""
    A, Solver = lib
    prob = W.config(name)
    orc = AFIETI(prob)
    s = Solver(prob, prec="fp64")
    try:
        assert s.n_c == orc.nc
        Bd = orc.B.toarray()
        X = np.eye(orc.ndof)
        for j in range(orc.ndof):
            y = s.apply(A.AFI_OP_B, T(X[j])).cpu().numpy()
            np.testing.assert_allclose(y, Bd[:, j], rtol=0, atol=1e-14)
        lam = np.random.default_rng(3).uniform(-1, 1, orc.nc)
        bt = s.apply(A.AFI_OP_BT, T(lam)).cpu().numpy()
        np.testing.assert_allclose(bt, orc.B.T @ lam, rtol=0, atol=1e-13)
    finally:
        s.close()


@pytest.mark.parametrize("prec", ["fp64", "tf32"])
@pytest.mark.parametrize("name,amp", POLY_CASES + [("NC3", np.array([1.0, -0.5, 0.75]))])
def test_gpu_reproduces_the_polynomial(lib, name, amp, prec):
    A, Solver = lib
    prob, u_ex, cf = polynomial_case(name, amp)
    s = Solver(prob, prec=prec, tol=1e-10, use_graph=True, maxit=4000)
    try:
        f = s.load_vector(cf)
        u, lam = s.solve(f)
        info = s.last_info
        un = u.cpu().numpy()
        assert info["relres_true"] <= 1e-10
        assert np.linalg.norm(un - u_ex) <= 1e-7 * np.linalg.norm(u_ex), \
            float(np.linalg.norm(un - u_ex) / np.linalg.norm(u_ex))
        # the continuity rows hold for the solution, and A u + B^T lambda = f
        bu = s.apply(A.AFI_OP_B, u).cpu().numpy()
        assert np.abs(bu).max() <= 1e-9 * np.abs(un).max()
        r = (f - s.apply(A.AFI_OP_STIFFNESS, u) - s.apply(A.AFI_OP_BT, lam)).cpu().numpy()
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(f.cpu().numpy())
        print(f"{name} {prec}: {info['iters']} iterations, u error "
              f"{np.linalg.norm(un - u_ex) / np.linalg.norm(u_ex):.1e}")
    finally:
        s.close()


def test_nested_face_with_a_free_edge_is_refused(lib):
    A, Solver = lib
    prob = W.config("NC3-small")
    df = prob.dirichlet_face.copy()
    df[1, 0] = 0            # patch 1's face eta_1 = 0 becomes natural: it meets both nested faces
    bad = dataclasses.replace(prob, dirichlet_face=df)
    with pytest.raises(A.AfiError):
        Solver(bad, prec="fp64")
