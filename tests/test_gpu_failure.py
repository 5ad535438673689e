"""The failure path of the tensor-core kernels, exercised without faulting the
GPU: a bounded mbarrier wait that nothing completes must run out, free its
tensor memory, return, and be reported as AFI_ETIMEOUT, after which the
context keeps working (afi_selftest_bounded_wait)."""
import numpy as np
import pytest

import afi_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_stays_usable():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti as A
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config("C2-small")
    s = Solver(prob, prec="tf32", tol=1e-8, local_only=True)
    try:
        x = torch.from_numpy(W.torn_random(prob, 5)[0]).cuda()
        before = s.fd(x)
        for polls in (1000, 20000):
            status, used = A.afi_selftest_bounded_wait(polls)
            assert status == A.AFI_ETIMEOUT
            assert used == polls
        after = s.fd(x)                      # tensor-core FD after the timeouts
        torch.cuda.synchronize()
        assert torch.equal(before, after)
        assert np.isfinite(after.cpu().numpy()).all()
    finally:
        s.close()
