"""All-Floating IETI (Section 4) with the inexact local solvers of Section 5.2
(or the exact ones of Section 5.1) and the non-redundant Schur preconditioner
of Remark 1, plus the conforming direct solve that defines the exact answer.  Oracle code: test infrastructure
only.

Readings where the paper is silent (each listed in the design notes):
  * B (Section 4, assumption ker B^T = 0): per component and per geometric node
    with copies c_1 < ... < c_m (ordered by (patch, local index)): a node on
    the Dirichlet boundary gets one row e_{c_j} per copy; any other node gets
    the star rows u_{c_1} - u_{c_j}, j = 2..m.  Rows are component-major, then
    nodes ordered by their first copy.
  * Nested non-conforming interfaces (Section 2; Section 6, non-conforming
    test): a face whose knot vectors refine the neighbouring patch's.  Its
    points off the Dirichlet boundary are not matched by coordinates; instead
    every such fine point f and component gets the row
    u_f - sum_c W[f, c] u_c over the coarse face points c off the Dirichlet
    boundary (W = the tensor product of the refinement matrices).  These rows
    follow all the node rows: faces by (fine patch, fine face), then
    component, then fine point.  The edges of a nested face must lie on the
    Dirichlet boundary.
  * lambda_0 = G (G^T G)^{-1} R^T f (minimum-norm choice of "such that").
  * H^(k) = diagonal of the bounding box of the patch control points.
  * P_A = P_A^inex (Section 5.2, plain parametric variant), P_S = the
    non-redundant form (B_G B_G^T)^{-1} B_G S_hat_H B_G^T (B_G B_G^T)^{-1} with
    S_hat_H = blkdiag H_k^{d-2} S_hat^(k) (Remark 1 with S replaced by S_hat).
  * MINRES stops when the preconditioned residual estimate has dropped by tol.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.spatial import cKDTree

from . import assembly, fd, nested
from .minres import minres


def _on_face(i_multi, ns, l, side):
    return i_multi[l] == (0 if side == 0 else ns[l] - 1)


class AFIETI:
    def __init__(self, prob, precond="inexact"):
        self.prob = prob
        self.dim = d = prob.dim
        self.np = prob.npatch
        self.geo = [assembly.PatchGeometry(prob.ctrl[k], prob.degree[k], prob.nel[k])
                    for k in range(self.np)]
        self.N = [int(np.prod(g.ns)) for g in self.geo]
        self.off = np.zeros(self.np + 1, dtype=np.int64)
        for k in range(self.np):
            self.off[k + 1] = self.off[k] + d * self.N[k]
        self.ndof = int(self.off[-1])
        # nested faces: (coarse patch, face, fine patch, face, fine points,
        # coarse points, weights), ordered by (fine patch, fine face)
        self.nested_faces = []
        for (kc, fc, kf, ff) in sorted(getattr(prob, "nested", []), key=lambda t: (t[2], t[3])):
            pf, pc, W = nested.face_map(prob, kc, fc, kf, ff)
            self.nested_faces.append((kc, fc, kf, ff, pf, pc, W))
        self._connectivity()
        self._constraints()
        self._rigid()
        self.A = None
        self.precond = precond

    # ------------------------------------------------------------------ nodes
    def _multi(self, k, i):
        ns = self.geo[k].ns
        out = []
        for n in ns:
            out.append(i % n)
            i //= n
        return out

    def _on_dirichlet(self, k, i):
        im = self._multi(k, i)
        return any(self.prob.dirichlet_face[k, f] and _on_face(im, self.geo[k].ns, f // 2, f % 2)
                   for f in range(2 * self.dim))

    def _connectivity(self):
        """Group shell control points of all patches into geometric nodes by
        coordinate matching (conforming, watertight interfaces, Section 2.2).
        Points of nested faces off the Dirichlet boundary stay single."""
        apart = set()
        for (kc, fc, kf, ff, pf, pc, W) in self.nested_faces:
            for k, pts_ in ((kc, pc), (kf, pf)):
                for i in pts_:
                    if not self._on_dirichlet(k, i):
                        apart.add((k, i))
        keys, pts, single = [], [], []
        for k, g in enumerate(self.geo):
            for i in range(self.N[k]):
                im = self._multi(k, i)
                if any(im[l] in (0, g.ns[l] - 1) for l in range(self.dim)):
                    if (k, i) in apart:
                        single.append([(k, i)])
                        continue
                    keys.append((k, i))
                    pts.append(g.X[i])
        pts = np.array(pts)
        scale = np.ptp(pts, axis=0).max()
        tree = cKDTree(pts)
        parent = list(range(len(keys)))

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a
        for a, b in tree.query_pairs(1e-10 * scale):
            ra, rb = find(a), find(b)
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
        groups = {}
        for a in range(len(keys)):
            groups.setdefault(find(a), []).append(keys[a])
        nodes = [sorted(v) for v in groups.values()] + single
        nodes.sort(key=lambda c: c[0])
        self.nodes = nodes
        self.dirichlet = []
        for copies in nodes:
            dn = False
            for (k, i) in copies:
                im = self._multi(k, i)
                for f in range(2 * self.dim):
                    if self.prob.dirichlet_face[k, f] and _on_face(im, self.geo[k].ns, f // 2, f % 2):
                        dn = True
            self.dirichlet.append(dn)

    def dof(self, k, c, i):
        return int(self.off[k] + c * self.N[k] + i)

    def _constraints(self):
        rows, cols, vals = [], [], []
        r = 0
        self.node_rows = []      # (component, node index, list of row ids)
        for c in range(self.dim):
            for n, copies in enumerate(self.nodes):
                ids = []
                if self.dirichlet[n]:
                    for (k, i) in copies:
                        rows.append(r); cols.append(self.dof(k, c, i)); vals.append(1.0)
                        ids.append(r); r += 1
                elif len(copies) >= 2:
                    k1, i1 = copies[0]
                    for (k, i) in copies[1:]:
                        rows += [r, r]
                        cols += [self.dof(k1, c, i1), self.dof(k, c, i)]
                        vals += [1.0, -1.0]
                        ids.append(r); r += 1
                self.node_rows.append((c, n, ids))
        # nested faces: u_f - sum_c W[f, c] u_c per free fine point
        self.nested_rows = []    # (component, fine patch, fine face, list of row ids)
        for (kc, fc, kf, ff, pf, pc, W) in self.nested_faces:
            cfree = [j for j, i in enumerate(pc) if not self._on_dirichlet(kc, i)]
            for c in range(self.dim):
                ids = []
                for a, i in enumerate(pf):
                    if self._on_dirichlet(kf, i):
                        continue
                    rows.append(r); cols.append(self.dof(kf, c, i)); vals.append(1.0)
                    for j in cfree:
                        if W[a, j] != 0.0:
                            rows.append(r); cols.append(self.dof(kc, c, pc[j])); vals.append(-W[a, j])
                    ids.append(r); r += 1
                self.nested_rows.append((c, kf, ff, ids))
        self.nc = r
        self.B = sp.csr_matrix((vals, (rows, cols)), shape=(self.nc, self.ndof))
        shell = np.zeros(self.ndof, dtype=bool)
        for copies in self.nodes:
            for (k, i) in copies:
                for c in range(self.dim):
                    shell[self.dof(k, c, i)] = True
        self.shell = shell
        self.BBt = (self.B @ self.B.T).tocsc()
        self.BBt_lu = spla.splu(self.BBt)

    def _rigid(self):
        blocks = [sp.csr_matrix(assembly.rigid_modes(g.X)) for g in self.geo]
        self.nm = blocks[0].shape[1]
        self.R = sp.block_diag(blocks, format="csr")
        self.G = (self.B @ self.R).tocsr()
        self.GtG = (self.G.T @ self.G).toarray()
        self.RtR = [(b.T @ b).toarray() for b in blocks]
        self.H = []
        for g in self.geo:
            ext = g.X.max(axis=0) - g.X.min(axis=0)
            self.H.append(float(np.sqrt((ext ** 2).sum())))

    # --------------------------------------------------------------- operators
    def assemble(self):
        if self.A is None:
            blocks = [sp.csr_matrix(assembly.stiffness(g, *self.prob.lame[k]))
                      for k, g in enumerate(self.geo)]
            self.A = sp.block_diag(blocks, format="csr")
        return self.A

    def mass(self, k):
        """The scalar mapped mass M^(k) (dense), computed once per patch."""
        if not hasattr(self, "_mass"):
            self._mass = {}
        if k not in self._mass:
            self._mass[k], _ = assembly.mass_block(self.geo[k])
        return self._mass[k]

    def load(self, coeffs):
        """f^(k) = M^(k) c^(k) stacked over patches."""
        return np.concatenate([assembly.load_from_coeffs(g, coeffs[k])
                               for k, g in enumerate(self.geo)])

    def P_chi(self, x):
        """Orthogonal projection onto ker(G^T) (eq. 4.6)."""
        return x - self.G @ np.linalg.solve(self.GtG, self.G.T @ x)

    def P_u(self, v):
        """Orthogonal projection onto range(A): I - R (R^T R)^{-1} R^T, patch-wise."""
        out = v.copy()
        for k in range(self.np):
            sl = slice(self.off[k], self.off[k + 1])
            Rk = self.R[sl][:, k * self.nm:(k + 1) * self.nm].toarray()
            out[sl] -= Rk @ np.linalg.solve(self.RtR[k], Rk.T @ v[sl])
        return out

    def _local(self):
        """Per patch and component: factorised H^{d-2}(A_hat_l + M_hat_l), the
        parametric A_hat_l and the factorised interior block (A_hat_l)_II."""
        if hasattr(self, "_loc"):
            return self._loc
        loc = []
        for k, g in enumerate(self.geo):
            lam, mu = self.prob.lame[k]
            Ks, Ms = fd.patch_1d(g.nel, g.p)
            mask = fd.interior_mask(g.ns)
            Hs = self.H[k] ** (self.dim - 2)
            per = []
            for l in range(self.dim):
                Ah = fd.A_hat(Ks, Ms, self.dim, l, lam, mu, sparse=True).tocsc()
                Mh = fd.M_hat(Ms, self.dim, sparse=True).tocsc()
                PA = spla.splu((Hs * (Ah + Mh)).tocsc())
                AII = spla.splu(Ah[mask][:, mask].tocsc())
                per.append((PA, Ah.tocsr(), AII))
            loc.append((per, mask, Hs))
        self._loc = loc
        return loc

    def PA_inv(self, r):
        """blkdiag_k,l [H^{d-2}(A_hat_l + M_hat_l)]^{-1} (eq. 5.6) by sparse LU."""
        out = np.empty_like(r)
        for k, (per, mask, Hs) in enumerate(self._local()):
            for l in range(self.dim):
                sl = slice(self.dof(k, l, 0), self.dof(k, l, 0) + self.N[k])
                out[sl] = per[l][0].solve(r[sl])
        return out

    def S_hat_H(self, t):
        """blkdiag_k H_k^{d-2} S_hat^(k) on a torn vector supported on the shell
        (eqs. 5.4-5.5, 5.7): S theta = A_GG theta - A_GI A_II^{-1} A_IG theta."""
        out = np.zeros_like(t)
        for k, (per, mask, Hs) in enumerate(self._local()):
            for l in range(self.dim):
                sl = slice(self.dof(k, l, 0), self.dof(k, l, 0) + self.N[k])
                Ah, AII = per[l][1], per[l][2]
                v = np.where(mask, 0.0, t[sl])
                y = Ah @ v
                vI = -AII.solve(y[mask])
                v2 = v.copy()
                v2[mask] = vI
                z = Ah @ v2
                out[sl] = np.where(mask, 0.0, Hs * z)
        return out

    def P_S(self, x):
        y = self.BBt_lu.solve(x)
        y = self.B @ self.S_hat_H(self.B.T @ y)
        return self.BBt_lu.solve(y)

    # ------------------------------------------------ exact local solvers
    def _exact(self):
        """Per patch (Section 5.1): the factorised P_A^ex = A^(k) + H_k^{-2} M^(k)
        (eq. 5.1 with D_H = H^{-2} I, the scalar mass on every component) and the
        factorised interior block A^(k)_II of the elasticity matrix (all
        components coupled), for the exact Schur complement S^(k)."""
        if hasattr(self, "_exa"):
            return self._exa
        A = self.assemble()
        out = []
        for k, g in enumerate(self.geo):
            sl = slice(self.off[k], self.off[k + 1])
            Ak = A[sl][:, sl].tocsc()
            Mk = self.mass(k)
            Md = sp.block_diag([sp.csr_matrix(Mk)] * self.dim)
            PA = spla.splu((Ak + Md / self.H[k] ** 2).tocsc())
            mask = np.tile(fd.interior_mask(g.ns), self.dim)
            AII = spla.splu(Ak[mask][:, mask].tocsc())
            out.append((PA, Ak.tocsr(), AII, mask))
        self._exa = out
        return out

    def PA_inv_exact(self, r):
        """blkdiag_k (A^(k) + H_k^{-2} M^(k))^{-1} r by sparse LU (eq. 5.1)."""
        out = np.empty_like(r)
        for k, (PA, _, _, _) in enumerate(self._exact()):
            sl = slice(self.off[k], self.off[k + 1])
            out[sl] = PA.solve(r[sl])
        return out

    def S_exact(self, t):
        """blkdiag_k S^(k) on a torn vector supported on the shell: the Schur
        complement of A^(k) on its interface dofs, S theta = (A v)_Gamma with
        v_Gamma = theta and v_I = -A_II^{-1} (A v^0)_I (Section 5.1)."""
        out = np.zeros_like(t)
        for k, (_, Ak, AII, mask) in enumerate(self._exact()):
            sl = slice(self.off[k], self.off[k + 1])
            v = np.where(mask, 0.0, t[sl])
            y = Ak @ v
            v[mask] = -AII.solve(y[mask])
            z = Ak @ v
            out[sl] = np.where(mask, 0.0, z)
        return out

    def P_S_exact(self, x):
        """P_S^{ex-nr} = (B B^T)^{-1} B S B^T (B B^T)^{-1} (Remark 1)."""
        y = self.BBt_lu.solve(x)
        y = self.B @ self.S_exact(self.B.T @ y)
        return self.BBt_lu.solve(y)

    # --------------------------------------- geometry-inclusion local solvers
    def _geo(self):
        """Per patch, the geometry-inclusion blocks of Section 5.2.3 (oracle/geo.py)."""
        if hasattr(self, "_geol"):
            return self._geol
        from . import geo
        A = self.assemble()
        out = []
        for k, g in enumerate(self.geo):
            sl = slice(self.off[k], self.off[k + 1])
            lam, mu = self.prob.lame[k]
            out.append(geo.GeoLocal(g, lam, mu, self.H[k], A[sl][:, sl].tocsr(), self.mass(k)))
        self._geol = out
        return out

    def PA_inv_geo(self, r):
        """blkdiag_{k,l} (P~_A^{inex,(k)})^{-1} r (eq. 5.12)."""
        out = np.empty_like(r)
        for k, gl in enumerate(self._geo()):
            for l in range(self.dim):
                sl = slice(self.dof(k, l, 0), self.dof(k, l, 0) + self.N[k])
                out[sl] = gl.PA_inv(l, r[sl])
        return out

    def S_geo(self, t):
        """blkdiag_{k,l} D_S^{1/2} S~_l D_S^{1/2} on a shell-supported torn vector (eq. 5.13)."""
        out = np.zeros_like(t)
        for k, gl in enumerate(self._geo()):
            for l in range(self.dim):
                sl = slice(self.dof(k, l, 0), self.dof(k, l, 0) + self.N[k])
                out[sl] = gl.S(l, t[sl])
        return out

    def P_S_geo(self, x):
        """P~_S^{inex-nr} = (B B^T)^{-1} B S~ B^T (B B^T)^{-1} (Remark 1)."""
        y = self.BBt_lu.solve(x)
        y = self.B @ self.S_geo(self.B.T @ y)
        return self.BBt_lu.solve(y)

    def precond_apply(self, rw, rc):
        """B^{-1} of eq. 4.9: blkdiag(P_u P_A^{-1} P_u^T, P_chi P_S P_chi^T), with
        the inexact local solvers (Section 5.2), or for precond="exact" the exact
        ones (Section 5.1), or for precond="geo" the geometry-inclusion ones
        (Section 5.2.3)."""
        if self.precond == "geo":
            zw = self.P_u(self.PA_inv_geo(self.P_u(rw)))
            zc = self.P_chi(self.P_S_geo(self.P_chi(rc)))
            return zw, zc
        if self.precond == "exact":
            zw = self.P_u(self.PA_inv_exact(self.P_u(rw)))
            zc = self.P_chi(self.P_S_exact(self.P_chi(rc)))
            return zw, zc
        zw = self.P_u(self.PA_inv(self.P_u(rw)))
        zc = self.P_chi(self.P_S(self.P_chi(rc)))
        return zw, zc

    def lambda0(self, f):
        return self.G @ np.linalg.solve(self.GtG, self.R.T @ f)

    def op(self, w, chi):
        """The projected saddle operator of eq. 4.7."""
        A = self.assemble()
        pc = self.P_chi(chi)
        return A @ w + self.B.T @ pc, self.P_chi(self.B @ w)

    def recover(self, w, chi, lam0):
        u = w - self.R @ np.linalg.solve(self.GtG, self.G.T @ (self.B @ w))
        return u, lam0 + chi

    def solve(self, f, tol=1e-8, maxit=2000, callback=None, check_true=True):
        """AF-IETI: MINRES on B^{-1} A (Section 4) then recovery of (u, lambda)."""
        self.assemble()
        lam0 = self.lambda0(f)
        n = self.ndof

        def Aop(x):
            a, b = self.op(x[:n], x[n:])
            return np.concatenate([a, b])

        def Mop(x):
            a, b = self.precond_apply(x[:n], x[n:])
            return np.concatenate([a, b])
        b = np.concatenate([f - self.B.T @ lam0, np.zeros(self.nc)])
        bn = np.linalg.norm(b)

        def true_rel(x):
            return float(np.linalg.norm(b - Aop(x)) / bn)
        x, info = minres(Aop, b, Mop, tol=tol, maxit=maxit, callback=callback,
                         true_check=true_rel if check_true else None)
        u, lam = self.recover(x[:n], x[n:], lam0)
        info["true_relres"] = float(np.linalg.norm(b - Aop(x)) / np.linalg.norm(b))
        return u, lam, info

    # ------------------------------------------------------- direct reference
    def conforming_basis(self):
        """Z: torn copies of every free (non-Dirichlet) global node/component;
        on a nested face the free fine points are not free: they follow the
        free coarse points with the weights W (the knot-insertion relation)."""
        rows, cols, vals = [], [], []
        col = 0
        shell_set = {}
        for n, copies in enumerate(self.nodes):
            for (k, i) in copies:
                shell_set[(k, i)] = n
        follows, fine_dep = {}, set()
        for (kc, fc, kf, ff, pf, pc, W) in self.nested_faces:
            for a, i in enumerate(pf):
                if self._on_dirichlet(kf, i):
                    continue
                fine_dep.add((kf, i))
                for j, ic in enumerate(pc):
                    if W[a, j] != 0.0 and not self._on_dirichlet(kc, ic):
                        follows.setdefault((kc, ic), []).append((kf, i, W[a, j]))
        for c in range(self.dim):
            for n, copies in enumerate(self.nodes):
                if self.dirichlet[n] or (len(copies) == 1 and copies[0] in fine_dep):
                    continue
                for (k, i) in copies:
                    rows.append(self.dof(k, c, i)); cols.append(col); vals.append(1.0)
                    for (kf, i2, w) in follows.get((k, i), []):
                        rows.append(self.dof(kf, c, i2)); cols.append(col); vals.append(w)
                col += 1
            for k in range(self.np):
                for i in range(self.N[k]):
                    if (k, i) not in shell_set:
                        rows.append(self.dof(k, c, i)); cols.append(col); vals.append(1.0)
                        col += 1
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.ndof, col))

    def direct_solve(self, f):
        """The conforming Galerkin solution of eq. 3.2 (unique by Section 4)
        and the multipliers from A u + B^T lambda = f."""
        A = self.assemble()
        Z = self.conforming_basis()
        K = (Z.T @ A @ Z).tocsc()
        ug = spla.spsolve(K, Z.T @ f)
        u = Z @ ug
        lam = self.BBt_lu.solve(self.B @ (f - A @ u))
        return u, lam
