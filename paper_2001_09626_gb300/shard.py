"""Patch-sharded AF-IETI over several GPUs, one process per GPU: the partition,
the exchange plan, the distributed operators built from per-rank local ones,
and the preconditioned MINRES driver (Section 4, eqs. 4.6, 4.7, 4.9).

The FETI subdomains are the patches, so the method shards by patch:
  * a rank owns a set of patches (their torn dofs, patch by patch in
    increasing patch order) and the constraint rows whose first copy lies on
    one of them.  All rows of a geometric node share that first copy, so the
    node-wise (B B^T)^{-1} of P_S (Remark 1) never crosses ranks;
  * B w needs, for each owned row whose second copy lives elsewhere, that
    copy's value: a point-to-point halo of shell values;
  * B^T chi sends the same rows' multipliers back the other way;
  * G^T chi = R^T B^T chi is a per-patch 6-vector (3 in 2D): an all-gather,
    after which every rank applies (G^T G)^{-1} redundantly;
  * MINRES inner products are an all-reduce of per-rank partial sums.

The patch-local pieces (stiffness A^(k), the local solvers P_A^{-1}, the Schur
block S^(k), the rigid modes R_k) come from the caller as callables acting on
a rank's own patches; on GPUs they are the library's kernels on a context
that holds those patches.  Exchanges use torch.distributed (NCCL across GPUs,
gloo on CPU).  The constraint rows are the library's (dof A, dof B or -1),
one star row u_A - u_B per additional copy of a node, or e_A for a copy on
the Dirichlet boundary (reading 1 of the design notes).  The rows of nested
non-conforming faces (a fine copy tied to several coarse ones with
knot-insertion weights) are not covered: a sharded form would give each
nested face's rows to the fine patch's owner and bring the coarse face's
values in by the same kind of halo."""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.distributed as dist


def lpt_partition(sizes, nranks):
    """Longest-processing-time assignment of patches (sizes = dofs per patch)
    to ranks: patches in decreasing size, each to the least loaded rank
    (lowest rank on ties).  Returns owner[patch]."""
    order = sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k))
    load = [0] * nranks
    owner = np.empty(len(sizes), dtype=np.int64)
    for k in order:
        r = min(range(nranks), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += int(sizes[k])
    return owner


class ExchangePlan:
    """What rank `rank` owns and exchanges, built identically on every rank
    from the global row list, the torn offsets of the patches and the owner
    of every patch."""

    def __init__(self, rows, offsets, owner, rank, nranks):
        rows = np.asarray(rows, dtype=np.int64)
        offsets = np.asarray(offsets, dtype=np.int64)
        self.rank, self.nranks = rank, nranks
        self.owner = np.asarray(owner, dtype=np.int64)
        npatch = len(offsets) - 1
        self.patches = [k for k in range(npatch) if self.owner[k] == rank]
        # local torn layout: own patches in increasing order
        self.loc_off = {}
        n = 0
        for k in self.patches:
            self.loc_off[k] = n
            n += int(offsets[k + 1] - offsets[k])
        self.n_local = n
        self.offsets = offsets

        def patch_of(d):
            return int(np.searchsorted(offsets, d, side="right") - 1)

        def local(d):
            k = patch_of(d)
            return self.loc_off[k] + int(d - offsets[k])
        pa = np.array([patch_of(d) for d in rows[:, 0]], dtype=np.int64)
        pb = np.array([patch_of(d) if d >= 0 else -1 for d in rows[:, 1]], dtype=np.int64)
        own = self.owner[pa] == rank
        self.rows = np.nonzero(own)[0]                    # owned global rows, increasing
        self.n_rows = len(self.rows)
        self.a_loc = np.array([local(d) for d in rows[self.rows, 0]], dtype=np.int64)
        # second copies: local, remote (halo) or none (Dirichlet row)
        self.b_loc = np.full(self.n_rows, -1, dtype=np.int64)
        self.halo_in = {}    # peer -> (positions among owned rows, peer's local dofs)
        for i, r in enumerate(self.rows):
            if rows[r, 1] < 0:
                continue
            q = int(self.owner[pb[r]])
            if q == rank:
                self.b_loc[i] = local(rows[r, 1])
            else:
                self.halo_in.setdefault(q, ([], []))
                self.halo_in[q][0].append(i)
                self.halo_in[q][1].append(int(rows[r, 1]))
        # rows owned elsewhere whose second copy is here: we send those copies'
        # values for B w and receive those rows' multipliers for B^T chi
        self.halo_out = {}   # peer -> local dofs (in the peer's row order)
        for r in np.nonzero(~own)[0]:
            if rows[r, 1] < 0 or self.owner[pb[r]] != rank:
                continue
            q = int(self.owner[pa[r]])
            self.halo_out.setdefault(q, []).append(local(rows[r, 1]))
        # (positions among the owned rows, global second copies), in increasing
        # row order on both sides of each exchange
        self.halo_in = {q: (np.array(p, dtype=np.int64), np.array(d, dtype=np.int64))
                        for q, (p, d) in self.halo_in.items()}
        self.halo_out = {q: np.array(v, dtype=np.int64) for q, v in self.halo_out.items()}
        # node groups of the owned star rows (consecutive rows sharing a first
        # copy) for the node-wise (B B^T)^{-1} = I - 1 1^T / m on each star
        self.groups = []
        i = 0
        while i < self.n_rows:
            j = i + 1
            if self.b_loc[i] >= 0 or i in self._halo_positions():
                while (j < self.n_rows and rows[self.rows[j], 0] == rows[self.rows[i], 0]
                       and rows[self.rows[j], 1] >= 0):
                    j += 1
                self.groups.append((i, j))
            i = j

    def _halo_positions(self):
        if not hasattr(self, "_hp"):
            self._hp = set()
            for p, _ in self.halo_in.values():
                self._hp.update(int(x) for x in p)
        return self._hp


def _exchange(send, recv_shapes, dtype, device):
    """Point-to-point: send[q] (1-D tensors) to each peer q, receive
    recv_shapes[q] values from each peer; returns {q: tensor}."""
    reqs, out = [], {}
    for q, n in sorted(recv_shapes.items()):
        out[q] = torch.empty(n, dtype=dtype, device=device)
        reqs.append(dist.irecv(out[q], src=q))
    for q, t in sorted(send.items()):
        reqs.append(dist.isend(t.contiguous(), dst=q))
    for r in reqs:
        r.wait()
    return out


class DistributedAFIETI:
    """The projected saddle operator of eq. 4.7, the preconditioner of eq. 4.9
    and MINRES on them, with torn vectors and multipliers split by the plan.

    local_ops must provide, for the rank's own patches in the plan's local
    layout (torch float64 tensors):
      A(w) -> A w;  PA_inv(r) -> P_A^{-1} r;  S(t) -> blkdiag S^(k) t
      (shell-supported in and out); Rt(w) -> [npatch_own, nm] of R_k^T w_k;
      R(y) -> R y for y [npatch_own, nm];  RtR_inv -> [npatch_own, nm, nm];
    and GtG_inv, the dense (G^T G)^{-1} over all patches (replicated)."""

    def __init__(self, plan, local_ops, GtG_inv, nm, device="cpu"):
        self.p = plan
        self.ops = local_ops
        self.GtG_inv = torch.as_tensor(GtG_inv, dtype=torch.float64, device=device)
        self.nm = nm
        self.dev = device
        self.npatch = len(plan.owner)

    # ---------------------------------------------------------- exchanges
    def B(self, w):
        """Owned rows of B w."""
        p = self.p
        out = w[torch.as_tensor(p.a_loc)].clone()
        bl = torch.as_tensor(p.b_loc)
        m = bl >= 0
        out[m] -= w[bl[m]]
        send = {q: w[torch.as_tensor(d)] for q, d in p.halo_out.items()}
        got = _exchange(send, {q: len(v[0]) for q, v in p.halo_in.items()}, w.dtype, w.device)
        for q, (pos, _) in p.halo_in.items():
            out[torch.as_tensor(pos)] -= got[q]
        return out

    def Bt(self, chi):
        """B^T chi on the rank's own dofs, from its owned rows' multipliers."""
        p = self.p
        w = torch.zeros(p.n_local, dtype=chi.dtype, device=chi.device)
        w.index_add_(0, torch.as_tensor(p.a_loc), chi)
        bl = torch.as_tensor(p.b_loc)
        m = bl >= 0
        w.index_add_(0, bl[m], -chi[m])
        send = {q: chi[torch.as_tensor(pos)] for q, (pos, _) in p.halo_in.items()}
        got = _exchange(send, {q: len(d) for q, d in p.halo_out.items()}, chi.dtype, chi.device)
        for q, d in p.halo_out.items():
            w.index_add_(0, torch.as_tensor(d), -got[q])
        return w

    def dot(self, a, b):
        s = torch.dot(a, b).reshape(1)
        dist.all_reduce(s)
        return float(s.item())

    def _gather_patch_vectors(self, g_own):
        """[npatch_own, nm] per rank -> [npatch, nm] on every rank."""
        n = torch.tensor([g_own.shape[0]], device=g_own.device)
        all_n = [torch.zeros_like(n) for _ in range(self.p.nranks)]
        dist.all_gather(all_n, n)
        mx = int(max(int(x) for x in all_n))
        pad = torch.zeros(mx, self.nm, dtype=g_own.dtype, device=g_own.device)
        pad[:g_own.shape[0]] = g_own
        parts = [torch.zeros_like(pad) for _ in range(self.p.nranks)]
        dist.all_gather(parts, pad)
        out = torch.zeros(self.npatch, self.nm, dtype=g_own.dtype, device=g_own.device)
        for q in range(self.p.nranks):
            ks = [k for k in range(self.npatch) if self.p.owner[k] == q]
            out[ks] = parts[q][:len(ks)]
        return out

    def Pchi(self, chi):
        """chi - G (G^T G)^{-1} G^T chi (eq. 4.6), G = B R."""
        return chi - self.B(self.ops.R(self._G_solve(self.ops.Rt(self.Bt(chi)))))

    def Pu(self, w):
        """w - R (R^T R)^{-1} R^T w, patch by patch (local)."""
        g = self.ops.Rt(w)
        y = torch.einsum("kab,kb->ka", self.ops.RtR_inv, g)
        return w - self.ops.R(y)

    def BBt_inv(self, chi):
        """Node-wise (B B^T)^{-1}: identity on Dirichlet rows, I - 1 1^T / m on
        each star of m - 1 rows (Remark 1)."""
        out = chi.clone()
        for a, b in self.p.groups:
            m = b - a + 1
            out[a:b] = chi[a:b] - chi[a:b].sum() / m
        return out

    def PS(self, chi):
        y = self.BBt_inv(chi)
        return self.BBt_inv(self.B(self.ops.S(self.Bt(y))))

    def saddle(self, w, chi):
        pc = self.Pchi(chi)
        return self.ops.A(w) + self.Bt(pc), self.Pchi(self.B(w))

    def precond(self, rw, rc):
        zw = self.Pu(self.ops.PA_inv(self.Pu(rw)))
        zc = self.Pchi(self.PS(self.Pchi(rc)))
        return zw, zc

    def _G_solve(self, g_own):
        """(G^T G)^{-1} applied to the gathered per-patch vectors; returns the
        rank's own patches' rows [npatch_own, nm]."""
        g = self._gather_patch_vectors(g_own)
        y = (self.GtG_inv @ g.reshape(-1)).reshape(self.npatch, self.nm)
        return y[torch.as_tensor(self.p.patches)]

    def rhs(self, f):
        """lambda_0 = G (G^T G)^{-1} R^T f on the owned rows and
        b = [f - B^T lambda_0; 0] (Section 4)."""
        lam0 = self.B(self.ops.R(self._G_solve(self.ops.Rt(f))))
        return f - self.Bt(lam0), torch.zeros(self.p.n_rows, dtype=f.dtype, device=f.device), lam0

    def recover(self, w, chi, lam0):
        """u = w - R (G^T G)^{-1} G^T B w, lambda = lambda_0 + chi."""
        u = w - self.ops.R(self._G_solve(self.ops.Rt(self.Bt(self.B(w)))))
        return u, lam0 + chi

    # ------------------------------------------------------------ solve
    def minres(self, bw, bc, tol=1e-8, maxit=2000):
        """Preconditioned MINRES (Paige-Saunders) from zero on
        [saddle] [w; chi] = [bw; bc]; stops when the preconditioned residual
        estimate has dropped by tol.  Returns (w, chi, iterations, history)."""
        def cat(a, b):
            return torch.cat([a, b])
        n = self.p.n_local
        split = lambda v: (v[:n], v[n:])

        def Aop(v):
            return cat(*self.saddle(*split(v)))

        def Mop(v):
            return cat(*self.precond(*split(v)))

        def dotv(a, b):
            return self.dot(a, b)
        b = cat(bw, bc)
        x = torch.zeros_like(b)
        r1 = b.clone()
        y = Mop(r1)
        beta1 = dotv(r1, y)
        if beta1 < 0:
            raise RuntimeError("indefinite preconditioner")
        beta1 = math.sqrt(beta1)
        if beta1 == 0.0:
            return split(x) + (0, [])
        oldb, beta, dbar, epsln, phibar = 0.0, beta1, 0.0, 0.0, beta1
        cs, sn = -1.0, 0.0
        w = torch.zeros_like(b)
        w2 = torch.zeros_like(b)
        r2 = r1.clone()
        hist = []
        it = 0
        while it < maxit:
            it += 1
            v = (1.0 / beta) * y
            y = Aop(v)
            if it >= 2:
                y = y - (beta / oldb) * r1
            alfa = dotv(v, y)
            y = y - (alfa / beta) * r2
            r1, r2 = r2, y
            y = Mop(r2)
            oldb, beta = beta, dotv(r2, y)
            if beta < 0:
                raise RuntimeError("indefinite preconditioner")
            beta = math.sqrt(beta)
            oldeps = epsln
            delta = cs * dbar + sn * alfa
            gbar = sn * dbar - cs * alfa
            epsln = sn * beta
            dbar = -cs * beta
            gamma = max(math.hypot(gbar, beta), 1e-300)
            cs, sn = gbar / gamma, beta / gamma
            phi = cs * phibar
            phibar = sn * phibar
            w1, w2 = w2, w
            w = (v - oldeps * w1 - delta * w2) / gamma
            x = x + phi * w
            rel = phibar / beta1
            hist.append(rel)
            if rel <= tol:
                break
        return split(x) + (it, hist)
