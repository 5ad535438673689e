"""Object wrapper around one libafieti context plus the autograd Function.

``Solver`` owns a context and the torch buffers a user needs; ``IetiSolve``
is a torch.autograd.Function whose forward is ``ieti_solve`` and whose
backward is ``ieti_solve_adjoint`` followed by ``afi_lame_grad`` (the saddle
matrix is symmetric and A^(k) is linear in the Lame values)."""
from __future__ import annotations

import numpy as np
import torch

from . import afieti as _a


class Solver:
    def __init__(self, problem, prec="fp64", tol=1e-8, maxit=2000, device=None, use_graph=False,
                 local_only=False, fd_slab=False, stencil_f64=False, force_restart=False,
                 exact=False, geo=False, fd_fixed=False, matrix_free=False):
        if not torch.cuda.is_available():
            raise RuntimeError("libafieti needs a CUDA device")
        self.device = torch.device(device or "cuda")
        self.problem = problem
        with torch.cuda.device(self.device):
            self._P = _a.Problem(problem)
            self.ctx = _a.af_ieti_setup(self._P, prec=prec, tol=tol, maxit=maxit,
                                        use_graph=use_graph,
                                        variant=(_a.AFI_VARIANT_LOCAL_ONLY if local_only else 0)
                                        | (_a.AFI_VARIANT_FD_SLAB if fd_slab else 0)
                                        | (_a.AFI_VARIANT_STENCIL_F64 if stencil_f64 else 0)
                                        | (_a.AFI_VARIANT_FORCE_RESTART if force_restart else 0)
                                        | (_a.AFI_VARIANT_EXACT if exact else 0)
                                        | (_a.AFI_VARIANT_GEO if geo else 0)
                                        | (_a.AFI_VARIANT_FD_FIXED if fd_fixed else 0)
                                        | (_a.AFI_VARIANT_MATRIX_FREE if matrix_free else 0))
        self.n_dof, self.n_c = _a.afi_sizes(self.ctx)
        self.last_info = None

    def close(self):
        if getattr(self, "ctx", None):
            _a.af_ieti_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros(self, n, batch=None):
        shape = (n,) if batch is None else (batch, n)
        return torch.zeros(shape, dtype=torch.float64, device=self.device)

    def set_precision(self, prec):
        _a.afi_set_precision(self.ctx, prec)

    def load_vector(self, coeffs):
        """f = M c for per-patch nodal coefficients (list of [d, ...] arrays or a
        torn tensor)."""
        if isinstance(coeffs, (list, tuple)):
            coeffs = torch.from_numpy(np.concatenate([c.reshape(-1) for c in coeffs])).to(self.device)
        f = self.zeros(self.n_dof)
        _a.afi_load_vector(self.ctx, coeffs.contiguous(), f)
        return f

    def apply(self, op, x):
        n_in = {_a.AFI_OP_B: self.n_dof, _a.AFI_OP_BT: self.n_c, _a.AFI_OP_PCHI: self.n_c,
                _a.AFI_OP_PS: self.n_c}.get(op, None)
        n_out = {_a.AFI_OP_B: self.n_c, _a.AFI_OP_BT: self.n_dof, _a.AFI_OP_PCHI: self.n_c,
                 _a.AFI_OP_PS: self.n_c, _a.AFI_OP_PRECOND: self.n_dof + self.n_c,
                 _a.AFI_OP_SADDLE: self.n_dof + self.n_c}.get(op, self.n_dof)
        y = self.zeros(n_out)
        _a.afi_apply(self.ctx, op, x.contiguous(), y)
        return y

    def fd(self, r, interior=False):
        """P_A^{-1} r (or the interior solves) for one vector or a batch [nrhs, n]."""
        s = torch.empty_like(r)
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        _a.fd_apply(self.ctx, 1 if interior else 0, r.contiguous(), s, nrhs)
        return s

    def solve(self, f, with_lambda=True, allow_not_converged=False):
        nrhs = 1 if f.dim() == 1 else f.shape[0]
        u = torch.empty_like(f)
        lam = self.zeros(self.n_c, None if f.dim() == 1 else nrhs) if with_lambda else None
        self.last_info = _a.ieti_solve(self.ctx, f.contiguous(), u, lam, nrhs,
                                       allow_not_converged=allow_not_converged)
        return u, lam

    def solve_adjoint(self, g):
        z = torch.empty_like(g)
        zl = self.zeros(self.n_c)
        self.last_info = _a.ieti_solve_adjoint(self.ctx, g.contiguous(), z, zl, 1)
        return z, zl

    def lame_grad(self, u, z):
        g = self.zeros(2 * self.problem.npatch)
        _a.afi_lame_grad(self.ctx, u.contiguous(), z.contiguous(), g)
        return g.view(-1, 2)


class IetiSolve(torch.autograd.Function):
    """u = IetiSolve.apply(f, lame, solver): differentiable in f and in the
    per-patch Lame values (lame is [npatch, 2] and must equal the values the
    solver was set up with; it carries the gradient only)."""

    @staticmethod
    def forward(ctx, f, lame, solver):
        u, _ = solver.solve(f, with_lambda=False)
        ctx.solver = solver
        ctx.save_for_backward(u)
        return u

    @staticmethod
    def backward(ctx, gu):
        (u,) = ctx.saved_tensors
        z, _ = ctx.solver.solve_adjoint(gu.contiguous())
        # dJ/df = z and dJ/dtheta = -z^T (dA/dtheta) u (returned by afi_lame_grad)
        return z, ctx.solver.lame_grad(u, z), None
