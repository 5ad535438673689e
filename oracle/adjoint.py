"""Adjoint solve and gradients (an addition to the paper's method: the paper
has no differentiation).  The saddle matrix [A B^T; B 0] is symmetric, so the
adjoint of the AF-IETI solve is the same solve with the objective gradient as
right-hand side; A^(k) is linear in (lambda_k, mu_k) (eq. 3.1), which gives
    dJ/dtheta = -z^T (dA/dtheta) u,   dJ/df = z.
For the compliance J = f^T u the adjoint state is z = u and dJ/df = 2u.
Oracle code: test infrastructure only."""
from __future__ import annotations

import numpy as np

from . import assembly


def lame_gradient(s, u, z):
    """[npatch, 2]: -(z_k^T A_lam^(k) u_k, z_k^T A_mu^(k) u_k)."""
    out = np.zeros((s.np, 2))
    for k, g in enumerate(s.geo):
        A_lam, A_mu, _ = assembly.stiffness_parts(g)
        sl = slice(s.off[k], s.off[k + 1])
        out[k, 0] = -(z[sl] @ (A_lam @ u[sl]))
        out[k, 1] = -(z[sl] @ (A_mu @ u[sl]))
    return out


def compliance_and_grads(s, f, direct=True, tol=1e-12):
    """J = f^T u with dJ/df = 2u and the per-patch Lame gradients."""
    if direct:
        u, _ = s.direct_solve(f)
    else:
        u, _, _ = s.solve(f, tol=tol)
    return float(f @ u), 2.0 * u, lame_gradient(s, u, u)


def lame_gradient_quadrature(g, u_k, z_k):
    """-(int div z div u, int 2 eps(z):eps(u)) over one patch by quadrature
    (the same quantities as z^T A_lam u and z^T A_mu u, Section 3 form, without
    forming the patch matrices)."""
    from . import assembly
    import scipy.sparse as sp
    Phi0, Phis, w, cols, det, Q = assembly._geometry_block(g, g.full_q(), g.full_c())
    d = g.dim
    wd = w * np.abs(det)
    uk = u_k.reshape(d, -1)
    zk = z_k.reshape(d, -1)
    # parametric gradients at the quadrature points, then physical ones
    gu = np.stack([np.stack([Phis[a] @ uk[l] for a in range(d)], -1) for l in range(d)], 1)
    gz = np.stack([np.stack([Phis[a] @ zk[l] for a in range(d)], -1) for l in range(d)], 1)
    Gu = np.einsum("qla,qax->qlx", gu, Q)
    Gz = np.einsum("qla,qax->qlx", gz, Q)
    du = np.einsum("qll->q", Gu)
    dz = np.einsum("qll->q", Gz)
    eu = 0.5 * (Gu + np.swapaxes(Gu, 1, 2))
    ez = 0.5 * (Gz + np.swapaxes(Gz, 1, 2))
    return -float(np.sum(wd * du * dz)), -float(np.sum(wd * 2.0 * np.einsum("qlx,qlx->q", eu, ez)))
