"""Patch-sharded AF-IETI over several GPUs, one process per GPU: the partition,
the exchange plan, the distributed operators built from per-rank local ones,
and the preconditioned MINRES driver (Section 4, eqs. 4.6, 4.7, 4.9).

The FETI subdomains are the patches, so the method shards by patch:
  * a rank owns a set of patches (their torn dofs, patch by patch in
    increasing patch order) and the constraint rows whose lead entry (below)
    lies on one of them.  All rows of a geometric node share that entry, and
    so do a nested face's rows, so the block-diagonal (B B^T)^{-1} of P_S
    (Remark 1) never crosses ranks;
  * B w needs, for each owned row with entries on patches owned elsewhere,
    those dofs' values: a point-to-point halo of shell values;
  * B^T chi sends the same rows' weighted multipliers back the other way;
  * G^T chi = R^T B^T chi is a per-patch 6-vector (3 in 2D): an all-gather,
    after which every rank applies (G^T G)^{-1} redundantly;
  * MINRES inner products are an all-reduce of per-rank partial sums.

The patch-local pieces (stiffness A^(k), the local solvers P_A^{-1}, the Schur
block S^(k), the rigid modes R_k) come from the caller as callables acting on
a rank's own patches; on GPUs they are the library's kernels on a context
that holds those patches.  Exchanges use torch.distributed (NCCL across GPUs,
gloo on CPU).  The constraint rows are the library's: one star row
u_A - u_B per additional copy of a node, or e_A for a copy on the Dirichlet
boundary, and the rows of nested non-conforming faces, which
tie a fine point to the coarse face's points with knot-insertion weights.
Any row belongs to the owner of its +1 entry (the first copy, or the fine
point), and its other entries are fetched by the halo; a nested face's rows
thus sit with the fine patch's owner, beside their dense (B B^T)^{-1}
block."""
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


def rows_csr(rows, ndof):
    """The constraint matrix B (scipy CSR) of star and Dirichlet rows given as
    (dof A, dof B or -1): u_A - u_B, or e_A."""
    import scipy.sparse as sp
    rows = np.asarray(rows, dtype=np.int64)
    r, c, v = [], [], []
    for i, (da, db) in enumerate(rows):
        r.append(i)
        c.append(int(da))
        v.append(1.0)
        if db >= 0:
            r.append(i)
            c.append(int(db))
            v.append(-1.0)
    return sp.csr_matrix((v, (r, c)), shape=(len(rows), int(ndof)))


class ExchangePlan:
    """What rank `rank` owns and exchanges, built identically on every rank
    from the global constraint rows, the torn offsets of the patches and the
    owner of every patch.

    rows is either an [n_c, 2] array (dof A, dof B or -1) of star and
    Dirichlet rows, or the constraint matrix B itself (scipy sparse, any
    rows).  A row belongs to the owner of its lead dof, the first entry with
    coefficient +1: the first copy of a node, or the fine point of a nested
    non-conforming face's row u_fine - sum_c W u_coarse.  Its other entries
    on patches owned elsewhere are the halo."""

    def __init__(self, rows, offsets, owner, rank, nranks):
        import scipy.sparse as sp
        from scipy.sparse.csgraph import connected_components
        offsets = np.asarray(offsets, dtype=np.int64)
        ndof = int(offsets[-1])
        if isinstance(rows, np.ndarray) or not sp.issparse(rows):
            B = rows_csr(rows, ndof)
        else:
            B = sp.csr_matrix(rows)
        B.sort_indices()
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
        patch_of = lambda d: np.searchsorted(offsets, d, side="right") - 1
        loc_base = np.full(npatch, -1, dtype=np.int64)
        for k in self.patches:
            loc_base[k] = self.loc_off[k] - offsets[k]
        ip, ix, dv = B.indptr, B.indices.astype(np.int64), B.data
        lead = np.empty(B.shape[0], dtype=np.int64)
        for r in range(B.shape[0]):
            pos = np.nonzero(dv[ip[r]:ip[r + 1]] == 1.0)[0]
            if len(pos) == 0:
                raise ValueError(f"constraint row {r} has no +1 entry")
            lead[r] = ix[ip[r] + pos[0]]
        row_owner = self.owner[patch_of(lead)]
        self.rows = np.nonzero(row_owner == rank)[0]          # owned global rows, increasing
        self.n_rows = len(self.rows)
        # entries of the owned rows: local (position, local dof, weight) and,
        # per peer, (position, slot among the peer's distinct dofs, weight)
        lp, ld, lw = [], [], []
        rem = {}
        for i, r in enumerate(self.rows):
            for e in range(ip[r], ip[r + 1]):
                d = int(ix[e])
                k = int(patch_of(d))
                q = int(self.owner[k])
                if q == rank:
                    lp.append(i)
                    ld.append(int(loc_base[k] + d))
                    lw.append(float(dv[e]))
                else:
                    rem.setdefault(q, []).append((i, d, float(dv[e])))
        self.loc_pos = np.array(lp, dtype=np.int64)
        self.loc_dof = np.array(ld, dtype=np.int64)
        self.loc_w = np.array(lw, dtype=np.float64)
        self.halo_in = {}    # peer -> (positions, slots, weights); the peer sends sorted dofs
        for q, ent in rem.items():
            dofs = np.unique(np.array([d for _, d, _ in ent], dtype=np.int64))
            slot = {int(d): j for j, d in enumerate(dofs)}
            self.halo_in[q] = (np.array([i for i, _, _ in ent], dtype=np.int64),
                               np.array([slot[d] for _, d, _ in ent], dtype=np.int64),
                               np.array([w for _, _, w in ent], dtype=np.float64), len(dofs))
        # rows owned elsewhere with entries on my patches: I send those dofs'
        # values for B w and receive their B^T contributions, in increasing
        # global dof order on both sides
        self.halo_out = {}   # peer -> my local dofs
        mine = np.zeros(npatch, dtype=bool)
        mine[self.patches] = True
        for r in np.nonzero(row_owner != rank)[0]:
            q = int(row_owner[r])
            for e in range(ip[r], ip[r + 1]):
                d = int(ix[e])
                k = int(patch_of(d))
                if mine[k]:
                    self.halo_out.setdefault(q, set()).add(d)
        self.halo_out = {q: np.array([int(loc_base[patch_of(d)] + d) for d in sorted(v)],
                                     dtype=np.int64) for q, v in self.halo_out.items()}
        # (B B^T)^{-1} of the owned rows: block diagonal over the connected
        # components of rows sharing a dof (a node's star; a nested face's
        # rows per component).  A component must not reach rows owned
        # elsewhere, which holds when every row touching a dof of an owned
        # row is owned here.
        Bo = B[self.rows]
        M = (Bo @ B.T).tocsr()
        if self.n_rows and np.any(row_owner[M.nonzero()[1]] != rank):
            raise ValueError("B B^T couples rows of two ranks: the node-wise block inverse "
                             "would cross ranks")
        Mo = (Bo @ Bo.T).tocsr()
        nb, lab = connected_components(Mo, directed=False) if self.n_rows else (0, np.zeros(0, int))
        self.blocks = []     # (positions, dense inverse of the block of B B^T)
        order = np.argsort(lab, kind="stable")
        starts = np.searchsorted(lab[order], np.arange(nb + 1))
        for b in range(nb):
            pos = order[starts[b]:starts[b + 1]]
            blk = Mo[pos][:, pos].toarray()
            self.blocks.append((pos, np.linalg.inv(blk)))


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
        out = torch.zeros(p.n_rows, dtype=w.dtype, device=w.device)
        out.index_add_(0, torch.as_tensor(p.loc_pos),
                       torch.as_tensor(p.loc_w) * w[torch.as_tensor(p.loc_dof)])
        send = {q: w[torch.as_tensor(d)] for q, d in p.halo_out.items()}
        got = _exchange(send, {q: v[3] for q, v in p.halo_in.items()}, w.dtype, w.device)
        for q, (pos, slot, wt, _) in p.halo_in.items():
            out.index_add_(0, torch.as_tensor(pos), torch.as_tensor(wt) * got[q][torch.as_tensor(slot)])
        return out

    def Bt(self, chi):
        """B^T chi on the rank's own dofs, from its owned rows' multipliers and
        the contributions of rows owned elsewhere."""
        p = self.p
        w = torch.zeros(p.n_local, dtype=chi.dtype, device=chi.device)
        w.index_add_(0, torch.as_tensor(p.loc_dof),
                     torch.as_tensor(p.loc_w) * chi[torch.as_tensor(p.loc_pos)])
        send = {}
        for q, (pos, slot, wt, nd) in p.halo_in.items():
            c = torch.zeros(nd, dtype=chi.dtype, device=chi.device)
            c.index_add_(0, torch.as_tensor(slot), torch.as_tensor(wt) * chi[torch.as_tensor(pos)])
            send[q] = c
        got = _exchange(send, {q: len(d) for q, d in p.halo_out.items()}, chi.dtype, chi.device)
        for q, d in p.halo_out.items():
            w.index_add_(0, torch.as_tensor(d), got[q])
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
        """(B B^T)^{-1} on the owned rows, block by block (Remark 1): on a
        node's star it is I - 1 1^T / m, on a nested face's rows the dense
        inverse of their block."""
        out = chi.clone()
        for pos, inv in self.p.blocks:
            pt = torch.as_tensor(pos)
            out[pt] = torch.as_tensor(inv, dtype=chi.dtype, device=chi.device) @ chi[pt]
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
