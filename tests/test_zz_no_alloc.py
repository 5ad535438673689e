"""The allocation-free FD entry point (for callers that may not allocate
device memory where they run a local solve: graph capture without allocation
nodes, fixed-budget real-time loops, plug-ins in frameworks that own all
device memory) against the context-based fd_apply.

It is fed eigen data computed on the host (scipy's generalised eigensolver
on the univariate matrices), so its eigenvector signs and order differ from
the library's own; Algorithm 1 does not depend on them.  The whole sweep
over all patch components runs twice in a row, which also exercises the
reuse of the shared static scratch.  Kept in its own file, collected last."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import fd as ofd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fd_apply_static_matches_fd_apply():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config("C2-small")
    s = Solver(prob, prec="fp64", tol=1e-8)
    try:
        r = torch.from_numpy(W.torn_random(prob, 21)[0]).cuda()
        ref = s.fd(r)
        off = prob.offsets()
        for sweep in range(2):
            out = torch.full_like(r, float("nan"))
            for k in range(prob.npatch):
                Ks, Ms = ofd.patch_1d(prob.nel[k], prob.degree[k])
                eig = [ofd.gen_eig(K, M) for K, M in zip(Ks, Ms)]
                U = [torch.from_numpy(np.ascontiguousarray(e[1])).cuda() for e in eig]
                D = [torch.from_numpy(np.ascontiguousarray(e[0])).cuda() for e in eig]
                X = prob.ctrl[k].reshape(-1, 3)
                H = float(np.sqrt(((X.max(0) - X.min(0)) ** 2).sum()))
                lam, mu = prob.lame[k]
                n = prob.n(k)
                N = int(np.prod(n))
                for l in range(3):
                    coef = [(2 * mu + lam) if j == l else mu for j in range(3)]
                    a = int(off[k]) + l * N
                    A.afi_fd_apply_static(n, U, D, coef, 1.0, H, r[a:a + N], out[a:a + N], 1)
            torch.cuda.synchronize()
            err = (out - ref).norm() / ref.norm()
            assert float(err) < 1e-10, (sweep, float(err))
        with pytest.raises(A.AfiError):
            big = torch.zeros(2 ** 20 + 8, dtype=torch.float64, device="cuda")
            A.afi_fd_apply_static((2 ** 20 + 8, 1, 1), [big, big], [big, big], [1, 1, 1], 1.0, 1.0,
                                  big, big, 1)
    finally:
        s.close()
