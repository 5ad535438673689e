"""GPU parity of the three-pass tensor-core FD (the path of tensors larger
than one CTA) against the CPU oracle, through the C ABI.

The context option AFI_VARIANT_FD_SLAB sends every 3D tensor through that
path, so it is checked here on patches the oracle solves quickly.  The
"uneven" shapes (14 x 13 x 16 and 11 x 13 x 16 basis functions) make the
plane groups (128 // 14 = 9 planes: 9 + 7) and the 128-line tiles of the
third-direction pass (182 lines: 128 + 54) end in a ragged tail; the
"aligned" shapes (12 x 12 x 14 and 16 x 12 x 14) take the vectorized loads.
Tolerances as in test_gpu_parity: TF32 1e-2, BF16 3e-2 per application, on every
(patch, component) block."""
import numpy as np
import pytest

import afi_workloads as W
from oracle.ieti import AFIETI

from blocks import block_rel, interior_blocks, torn_blocks

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


# (a) odd and even row lengths, plane sizes not multiples of 4: scalar and
#     two-wide loads; (b) rows and planes multiples of 4 (12x12x14, 16x12x14):
#     four-wide plane loads and 16-byte line loads
SHAPES = {"uneven": [[12, 9], [11], [14]], "aligned": [[10, 14], [10], [12]]}


@pytest.fixture(scope="module", params=sorted(SHAPES))
def slab(request):
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300.solver import Solver
    prob = W.quarter_annulus((2, 1, 1), 2, nel_cols=SHAPES[request.param], name="annulus-slab")
    orc = AFIETI(prob)
    s = Solver(prob, prec="tf32", tol=1e-8, local_only=True, fd_slab=True)
    ref = Solver(prob, prec="tf32", tol=1e-8, local_only=True)
    yield prob, orc, s, ref
    s.close()
    ref.close()


@pytest.mark.parametrize("prec,tol", [("tf32", 1e-2), ("bf16", 3e-2)])
def test_slab_fd_matches_oracle(slab, prec, tol):
    prob, orc, s, _ = slab
    s.set_precision(prec)
    x = W.torn_random(prob, 31)[0]
    y = s.fd(T(x)).cpu().numpy()
    assert block_rel(y, orc.PA_inv(x), torn_blocks(orc)) < tol


@pytest.mark.parametrize("prec,tol", [("tf32", 1e-2), ("bf16", 3e-2)])
def test_slab_interior_fd_matches_oracle(slab, prec, tol):
    prob, orc, s, _ = slab
    s.set_precision(prec)
    rng = np.random.default_rng(32)
    blocks, refs = [], []
    for per, mask, _ in orc._local():
        for l in range(orc.dim):
            r = rng.uniform(-1, 1, int(mask.sum()))
            blocks.append(r)
            refs.append(per[l][2].solve(r))
    out = s.fd(T(np.concatenate(blocks)), interior=True).cpu().numpy()
    assert block_rel(out, np.concatenate(refs), interior_blocks(orc)) < tol


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_slab_close_to_single_cta_path(slab, prec):
    """Both tensor-core paths compute the same products in the same operand
    precision; they differ in rounding order and the FP32 scratch only."""
    prob, _, s, ref = slab
    s.set_precision(prec)
    ref.set_precision(prec)
    x = T(W.torn_random(prob, 33)[0])
    a, b = s.fd(x), ref.fd(x)
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) < (5e-3 if prec == "tf32" else 3e-2)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_slab_batched_rhs_and_special_values(slab, prec):
    prob, orc, s, _ = slab
    s.set_precision(prec)
    R = T(W.torn_random(prob, 34, nrhs=3))
    batch = s.fd(R)
    for j in range(3):
        assert torch.equal(batch[j], s.fd(R[j].contiguous()))
    x = W.torn_random(prob, 35)[0]
    assert np.all(s.fd(T(np.zeros_like(x))).cpu().numpy() == 0.0)
    y = s.fd(T(x)).cpu().numpy()
    assert np.array_equal(s.fd(T(np.ldexp(x, 12))).cpu().numpy(), np.ldexp(y, 12))
    k, lo = 1, int(orc.off[1])                 # component 0 of patch 1
    hi = lo + orc.N[k]
    xn = x.copy()
    xn[lo + 5] = np.nan
    yn = s.fd(T(xn)).cpu().numpy()
    assert np.all(np.isnan(yn[lo:hi]))
    assert np.array_equal(yn[:lo], y[:lo]) and np.array_equal(yn[hi:], y[hi:])
