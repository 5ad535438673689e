"""The paper's weak-scalability experiment (Section 6, Table 3) on the GPU:
the unit cube split into N_patch = 2^3 ... 6^3 equal cubes, p = 3, 8
elements per direction and patch, natural conditions on x = 0 and x = 1,
Dirichlet elsewhere, geometry-inclusion local solvers (the paper's INEXACT)
and, where the dense per-patch inverses fit, the EXACT ones.

The paper's right-hand side comes from a manufactured solution with
inhomogeneous Dirichlet data; here the same solution's components are nodal
body-force coefficients with homogeneous data, and the library stops only
when the true residual also reaches 1e-8 (the paper stops on the MINRES
estimate).  So the counts are compared with the paper's within a band, and
what the table shows is checked directly: the iteration count stays flat as
N_patch grows (within 20% of the 2^3 count up to 6^3), and EXACT needs
fewer iterations than INEXACT.  The 2^3 count must also match the oracle's
with the same stopping rule (within 5%)."""
import os

import numpy as np
import pytest

import afi_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HERE = os.path.join(os.path.dirname(__file__), "golden")


def paper_rows():
    rows = {}
    for ln in open(os.path.join(HERE, "paper_table3.txt")):
        if ln.strip() and not ln.startswith("#"):
            n, ex, inex = map(int, ln.split())
            rows[n] = (ex, inex)
    return rows


def cube(n):
    P = W.with_neumann(W.unit_box(3, (n, n, n), 3, 8, name=f"cube-{n}^3-p3-n8"), (0, 1))
    coeffs = []
    for k in range(P.npatch):
        X = P.ctrl[k].reshape(-1, 3)
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        coeffs.append(np.stack([np.cos(x), z * np.sin(y), (x * y * z) ** 2]))
    return P, coeffs


def gpu_iters(P, coeffs, **kw):
    from paper_2001_09626_gb300.solver import Solver
    s = Solver(P, tol=1e-8, use_graph=True, maxit=4000, **kw)
    try:
        f = s.load_vector(coeffs)
        s.solve(f)
        info = s.last_info
        assert info["relres_true"] <= 1e-8
        return info["iters"]
    finally:
        s.close()


def test_table3_weak_scaling_on_gpu():
    import __graft_entry__ as g
    g.build()
    rows = paper_rows()
    its = {}
    for n in (2, 3, 4, 5, 6):
        P, coeffs = cube(n)
        its[n] = {"geo_tf32": gpu_iters(P, coeffs, prec="tf32", geo=True)}
        if n <= 3:
            its[n]["exact"] = gpu_iters(P, coeffs, exact=True)
        print(f"N_patch={n ** 3}: GPU {its[n]}  paper EXACT/INEXACT {rows[n ** 3]}")
    base = its[2]["geo_tf32"]
    for n in (3, 4, 5, 6):
        assert its[n]["geo_tf32"] <= 1.2 * base, its
    for n in (2, 3):
        assert its[n]["exact"] < its[n]["geo_tf32"], its
        ex, inex = rows[n ** 3]
        assert 0.8 * ex <= its[n]["exact"] <= 1.6 * ex, its
        assert 0.8 * inex <= its[n]["geo_tf32"] <= 1.5 * inex, its


def test_table3_first_row_matches_oracle():
    """N_patch = 2^3 with the geometry-inclusion solvers: GPU (FP64) and oracle,
    same stopping rule (estimate and true residual)."""
    import __graft_entry__ as g
    g.build()
    from oracle.ieti import AFIETI
    P, coeffs = cube(2)
    o = AFIETI(P, precond="geo")
    _, _, info = o.solve(o.load(coeffs), tol=1e-8)
    it = gpu_iters(P, coeffs, prec="fp64", geo=True)
    assert abs(it - info["iters"]) <= max(2, 0.05 * info["iters"]), (it, info["iters"])
