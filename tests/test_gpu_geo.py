"""Geometry-inclusion local solvers (Section 5.2.3, eqs. 5.11-5.13) on the GPU
(AFI_VARIANT_GEO) against the oracle's (oracle/geo.py, precond="geo").

The GPU fits the separable factors itself (same Diliberto-Straus sweeps,
same stopping rule); its targets differ from the oracle's by rounding, so
the fitted factors, and with them every operator, agree to about 1e-13.
FP64 operators are compared per block at 1e-9, the reduced-precision local
solvers at the tolerances of test_gpu_parity (they change only the
arithmetic of Algorithm 1, not the matrices), solves against the direct
solve at 1e-7.  The FP64 iteration count must be within 5% of the oracle's
with the same preconditioner, and on the curved annulus well below the
plain parametric solvers' count, which is what the variant is for."""
import numpy as np
import pytest

import afi_workloads as W
from oracle.ieti import AFIETI

from blocks import block_rel, interior_blocks, mult_blocks, saddle_blocks, torn_blocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = ["C1-small", "C2-small", "C4-small", "C5-small"]
PREC_TOL = {"fp64": 1e-9, "fp32": 2e-5, "tf32": 1e-2, "bf16": 3e-2}


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.fixture(scope="module", params=CASES)
def case(request):
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config(request.param)
    orc = AFIETI(prob, precond="geo")
    orc.assemble()
    orc._geo()
    s = Solver(prob, prec="fp64", tol=1e-10, geo=True)
    yield request.param, prob, orc, s
    s.close()


def test_geo_operators_fp64(case):
    from paper_2001_09626_gb300 import afieti as A
    _, prob, orc, s = case
    x = W.torn_random(prob, 71)[0]
    assert block_rel(s.apply(A.AFI_OP_PA_INV, T(x)).cpu().numpy(), orc.PA_inv_geo(x),
                     torn_blocks(orc)) < 1e-9
    t = W.torn_random(prob, 72)[0] * orc.shell
    assert block_rel(s.apply(A.AFI_OP_SCHUR, T(t)).cpu().numpy(), orc.S_geo(t),
                     torn_blocks(orc)) < 1e-9
    lam = np.random.default_rng(73).uniform(-1, 1, orc.nc)
    assert block_rel(s.apply(A.AFI_OP_PS, T(lam)).cpu().numpy(), orc.P_S_geo(lam),
                     mult_blocks(orc)) < 1e-9
    z = np.random.default_rng(74).uniform(-1, 1, orc.ndof + orc.nc)
    ref = np.concatenate(orc.precond_apply(z[:orc.ndof], z[orc.ndof:]))
    assert block_rel(s.apply(A.AFI_OP_PRECOND, T(z)).cpu().numpy(), ref, saddle_blocks(orc)) < 1e-9


@pytest.mark.parametrize("prec", list(PREC_TOL))
def test_geo_local_solvers(case, prec):
    """P~_A^{-1} and the interior solves (A~_l)_II^{-1} at every precision."""
    _, prob, orc, s = case
    s.set_precision(prec)
    try:
        x = W.torn_random(prob, 75)[0]
        assert block_rel(s.fd(T(x)).cpu().numpy(), orc.PA_inv_geo(x), torn_blocks(orc)) \
            < PREC_TOL[prec]
        rng = np.random.default_rng(76)
        blocks, refs = [], []
        for gl in orc._geo():
            for l in range(orc.dim):
                r = rng.uniform(-1, 1, int(gl.mask.sum()))
                blocks.append(r)
                refs.append(gl.per[l]["AII"].solve(r))
        out = s.fd(T(np.concatenate(blocks)), interior=True).cpu().numpy()
        assert block_rel(out, np.concatenate(refs), interior_blocks(orc)) < PREC_TOL[prec]
    finally:
        s.set_precision("fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_geo_solve(case, prec):
    name, prob, orc, s = case
    s.set_precision(prec)
    try:
        f = orc.load(W.body_force_coeffs(prob))
        u, lam = s.solve(T(f))
        info = s.last_info
        ud, ld = orc.direct_solve(f)
        assert info["relres_true"] <= 1e-10
        assert block_rel(u.cpu().numpy(), ud, torn_blocks(orc)) < 1e-7
        assert block_rel(lam.cpu().numpy(), ld, mult_blocks(orc)) < 1e-7
        if not hasattr(orc, "_test_iters"):
            orc._test_iters = orc.solve(f, tol=1e-10)[2]["iters"]
        oit = orc._test_iters
        if prec == "fp64":
            assert abs(info["iters"] - oit) <= max(2, 0.05 * oit), (info["iters"], oit)
        else:
            assert info["iters"] <= 1.1 * oit + 2, (info["iters"], oit)
    finally:
        s.set_precision("fp64")


def test_geo_beats_plain_on_the_annulus():
    """On the curved quarter annulus the plain parametric solvers lose most;
    the geometry-inclusion ones must need clearly fewer iterations (the
    oracle: 103 against 223 on this discretisation)."""
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = W.config("C4-small")
    coeffs = W.body_force_coeffs(prob)
    its = {}
    for geo in (False, True):
        s = Solver(prob, prec="tf32", tol=1e-8, geo=geo, use_graph=True)
        try:
            s.solve(s.load_vector(coeffs))
            its[geo] = s.last_info["iters"]
        finally:
            s.close()
    assert its[True] < 0.6 * its[False], its


def test_geo_rejects_incompatible_variants():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti as A
    prob = W.config("C1-small")
    for v in (A.AFI_VARIANT_LOCAL_ONLY, A.AFI_VARIANT_EXACT):
        with pytest.raises(A.AfiError):
            A.af_ieti_setup(prob, variant=A.AFI_VARIANT_GEO | v)
