"""The allocation-free FD entry point, afi_fd_apply_static.

It exists for callers that may not allocate device memory where they run a
local solve: code recorded into a CUDA graph that must hold no allocation
node, real-time loops on a fixed memory budget, or plug-ins whose host
framework owns every device byte.  Its intermediate tensors live in a fixed
file-scope device array instead.

Checks:
  * against the context-based fd_apply on every (patch, component) block of
    C2-small, over two sweeps in a row (the shared scratch is reused);
  * directly against the oracle's Algorithm 1 (tensordot FD) on a 2D shape
    and on a ragged 3D shape with several tensors per call, per tensor;
  * no device memory is taken by a call once the library is loaded;
  * invalid dimension data and oversized requests (including sizes whose
    product would overflow 64 bits) return AFI_EINVAL without running.

The eigen data come from the host (scipy's generalised eigensolver on the
oracle's univariate matrices), so eigenvector signs and order differ from
the library's own; the FD result does not depend on them.  Kept in its own
file, collected last."""
import numpy as np
import pytest

import afi_workloads as W
from oracle import fd as ofd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    import __graft_entry__ as g
    g.build()
    from paper_2001_09626_gb300 import afieti as A
    return A


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _blockrel(a, b, nblk):
    a = a.reshape(nblk, -1)
    b = b.reshape(nblk, -1)
    return max(float(np.linalg.norm(a[j] - b[j]) / np.linalg.norm(b[j])) for j in range(nblk))


def test_fd_apply_static_matches_fd_apply():
    A = _lib()
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
                U = [_cuda(e[1]) for e in eig]
                D = [_cuda(e[0]) for e in eig]
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
            o, rf = out.cpu().numpy(), ref.cpu().numpy()
            for k in range(prob.npatch):
                N = int(np.prod(prob.n(k)))
                for l in range(3):
                    a = int(off[k]) + l * N
                    e = np.linalg.norm(o[a:a + N] - rf[a:a + N]) / np.linalg.norm(rf[a:a + N])
                    assert e < 1e-10, (sweep, k, l, e)
    finally:
        s.close()


@pytest.mark.parametrize("nel,p,nblk,coef,shift,scale", [
    ((13, 6), 3, 3, (1.7, 0.4, 0.0), 1.0, 1.0),          # 2D, ragged rows
    ((9, 14, 5), 2, 4, (0.38, 1.3, 0.38), 1.0, 0.83),    # 3D, every extent different
    ((9, 14, 5), 2, 2, (0.5, 0.5, 1.6), 0.0, 1.0),       # 3D interior form (no shift)
])
def test_fd_apply_static_matches_oracle(nel, p, nblk, coef, shift, scale):
    """Each tensor against the oracle's FD (Algorithm 1 by tensordot) with the
    same Lambda; the interior case uses the pencils without their first and
    last index."""
    A = _lib()
    dim = len(nel)
    Ks, Ms = ofd.patch_1d(list(nel), p)
    if shift == 0.0:
        Ks = [ofd.interior(K) for K in Ks]
        Ms = [ofd.interior(M) for M in Ms]
    eig = [ofd.gen_eig(K, M) for K, M in zip(Ks, Ms)]
    n = [K.shape[0] for K in Ks]
    lamd = np.full([n[j] for j in reversed(range(dim))], shift)
    for j in range(dim):
        shape = [1] * dim
        shape[dim - 1 - j] = n[j]
        lamd = lamd + coef[j] * eig[j][0].reshape(shape)
    lamd = scale * lamd
    rng = np.random.default_rng(31)
    R = rng.uniform(-1, 1, (nblk,) + tuple(reversed(n)))
    ref = np.stack([ofd.fd_solve(R[b], [e[1] for e in eig], lamd) for b in range(nblk)])
    U = [_cuda(e[1]) for e in eig] + ([None] if dim == 2 else [])
    D = [_cuda(e[0]) for e in eig] + ([None] if dim == 2 else [])
    shape3 = tuple(n) + ((1,) if dim == 2 else ())
    r = _cuda(R.reshape(-1))
    for call in range(2):
        s = torch.full_like(r, float("nan"))
        A.afi_fd_apply_static(shape3, U, D, coef, shift, scale, r, s, nblk)
        torch.cuda.synchronize()
        assert _blockrel(s.cpu().numpy(), ref.reshape(-1), nblk) < 1e-11, call


def test_fd_apply_static_allocates_nothing():
    """Once the library's module is loaded (first call), further calls leave
    the device's free memory unchanged."""
    A = _lib()
    n = (12, 11, 10)
    Ks, Ms = ofd.patch_1d([n[0] - 2, n[1] - 2, n[2] - 2], 2)
    eig = [ofd.gen_eig(K, M) for K, M in zip(Ks, Ms)]
    U = [_cuda(e[1]) for e in eig]
    D = [_cuda(e[0]) for e in eig]
    r = _cuda(np.random.default_rng(5).uniform(-1, 1, 4 * int(np.prod(n))))
    s = torch.empty_like(r)
    A.afi_fd_apply_static(n, U, D, (1.0, 1.0, 1.0), 1.0, 1.0, r, s, 4)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        A.afi_fd_apply_static(n, U, D, (1.0, 1.0, 1.0), 1.0, 1.0, r, s, 4)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_fd_apply_static_rejects_bad_requests():
    A = _lib()
    big = torch.zeros(2 ** 20 + 8, dtype=torch.float64, device="cuda")
    one = torch.ones(4, dtype=torch.float64, device="cuda")
    # 2 * n1 > 2^21 doubles of scratch
    with pytest.raises(A.AfiError):
        A.afi_fd_apply_static((2 ** 20 + 8, 1, 1), [big, big], [big, big], [1, 1, 1], 1.0, 1.0,
                              big, big, 1)
    # dimensions whose product wraps a signed 64-bit integer
    h = 2 ** 31 - 1
    with pytest.raises(A.AfiError):
        A.afi_fd_apply_static((h, h, h), [one, one, one], [one, one, one], [1, 1, 1], 1.0, 1.0,
                              one, one, h)
    # n3 > 1 without third-direction data; third-direction U without D
    with pytest.raises(A.AfiError):
        A.afi_fd_apply_static((2, 2, 2), [one, one, None], [one, one, None], [1, 1, 1], 1.0, 1.0,
                              one, one, 1)
    with pytest.raises(A.AfiError):
        A.afi_fd_apply_static((2, 2, 1), [one, one, one], [one, one, None], [1, 1, 1], 1.0, 1.0,
                              one, one, 1)
