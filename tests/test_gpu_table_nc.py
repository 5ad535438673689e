"""The paper's non-conforming test (Section 6) on the GPU: the box
(0,1) x (0,3) x (0,1) in three patches with 4, 8 and 16 elements per
direction, nested interfaces, p = 1 .. 4, INEXACT local solvers (FP64 and
TF32 operands).

As in test_gpu_table3.py the right-hand side takes the paper's manufactured
solution's components as nodal body-force coefficients with homogeneous
Dirichlet data, and the library also stops on the true residual, so the
counts are compared with the paper's within a band: 10% with FP64 local
solvers (measured 85 / 94 / 99 / 105 against the paper's 86 / 96 / 104 /
111), -10% .. +15% with TF32 operands (measured 94 / 100 / 110 / 114).  What
the table shows is checked directly too: the iteration count depends only
mildly on p (the p = 4 count within 1.5x of the p = 1 count; the paper has
111 / 86 = 1.29)."""
import os

import numpy as np
import pytest

import afi_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HERE = os.path.join(os.path.dirname(__file__), "golden")


def paper_rows():
    rows = {}
    for ln in open(os.path.join(HERE, "paper_table_nonconforming.txt")):
        if ln.strip() and not ln.startswith("#"):
            p, ex, inex = map(int, ln.split())
            rows[p] = (ex, inex)
    return rows


def box(p):
    P = W.nested_box(3, (4, 8, 16), p, name=f"nc-box-p{p}")
    coeffs = []
    for k in range(P.npatch):
        X = P.ctrl[k].reshape(-1, 3)
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        coeffs.append(np.stack([np.cos(x), z * np.sin(y), (x * y * z) ** 2]))
    return P, coeffs


def test_nonconforming_table_on_gpu():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    rows = paper_rows()
    got = {}
    for prec in ("fp64", "tf32"):
        for p in sorted(rows):
            P, coeffs = box(p)
            s = Solver(P, prec=prec, tol=1e-8, use_graph=True, maxit=4000)
            try:
                f = s.load_vector(coeffs)
                s.solve(f)
                info = s.last_info
                assert info["relres_true"] <= 1e-8
                got[(prec, p)] = info["iters"]
            finally:
                s.close()
    print("p, paper INEXACT, GPU fp64, GPU tf32:",
          [(p, rows[p][1], got[("fp64", p)], got[("tf32", p)]) for p in sorted(rows)])
    for p in rows:
        # FP64 local solvers: the paper's method; TF32 operands may cost a few more
        assert abs(got[("fp64", p)] - rows[p][1]) <= 0.1 * rows[p][1], (p, got)
        assert 0.9 * rows[p][1] <= got[("tf32", p)] <= 1.15 * rows[p][1], (p, got)
    for prec in ("fp64", "tf32"):
        assert got[(prec, 4)] <= 1.5 * got[(prec, 1)], got
