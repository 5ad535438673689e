"""Nested non-conforming interfaces (Section 2): where the knot vector of one
patch refines the adjacent patch's, the coarse side's splines are linear
combinations of the fine side's, and the gluing rows of B tie every free fine
interface coefficient to that combination of the coarse ones (Section 6,
"non-conforming test": the knot-insertion property).  Oracle code: test
infrastructure only.

The refinement matrix E (fine coefficients = E @ coarse coefficients) is
computed here as the exact L2 projection of the coarse basis onto the fine
space, E = M_ff^{-1} M_fc with Gauss quadrature on the fine spans (exact:
the coarse splines are polynomials of degree p on every fine span).  It is
not the knot-insertion recursion: the two agree because the coarse space is
contained in the fine one.
"""
from __future__ import annotations

import numpy as np

from . import spline


def refinement_matrix(nel_c: int, nel_f: int, p: int) -> np.ndarray:
    """E [nel_f + p, nel_c + p] with b_c(x) = b_f(x) @ E for the open uniform
    knot vectors of nel_c and nel_f elements (nel_f a multiple of nel_c)."""
    if nel_f % nel_c:
        raise ValueError("the fine knot vector must refine the coarse one")
    kf, kc = spline.open_knots(nel_f, p), spline.open_knots(nel_c, p)
    x, w, _ = spline.quadrature(kf, p)
    Bf = spline.basis(kf, p, x)
    Bc = spline.basis(kc, p, x)
    Mff = Bf.T @ (w[:, None] * Bf)
    Mfc = Bf.T @ (w[:, None] * Bc)
    return np.linalg.solve(Mff, Mfc)


def face_points(ns, face):
    """Local indices (i1 fastest, increasing) of the control points of the
    face `face` = 2*l + side of a patch with basis counts ns, and for each its
    indices along the tangential directions (increasing direction order)."""
    dim = len(ns)
    l, side = divmod(face, 2)
    tang = [t for t in range(dim) if t != l]
    pts, tidx = [], []
    for i in range(int(np.prod(ns))):
        im, r = [], i
        for n in ns:
            im.append(r % n)
            r //= n
        if im[l] == (0 if side == 0 else ns[l] - 1):
            pts.append(i)
            tidx.append(tuple(im[t] for t in tang))
    return pts, tidx, tang


def face_map(prob, kc, fc, kf, ff):
    """The weights of a nested face: for every fine face point (in increasing
    local index) the dense row of E_{t1} (x) E_{t2} over the coarse face
    points (in increasing local index).  Returns (fine points, coarse points,
    W [n fine, n coarse])."""
    nsc, nsf = prob.n(kc), prob.n(kf)
    p = int(prob.degree[kc])
    if int(prob.degree[kf]) != p:
        raise ValueError("nested faces need one degree")
    pc, tc, tang_c = face_points(nsc, fc)
    pf, tf, tang_f = face_points(nsf, ff)
    Es = [refinement_matrix(int(prob.nel[kc, a]), int(prob.nel[kf, b]), p)
          for a, b in zip(tang_c, tang_f)]
    W = np.ones((len(pf), len(pc)))
    for t, E in enumerate(Es):
        fi = np.array([q[t] for q in tf])
        ci = np.array([q[t] for q in tc])
        W *= E[np.ix_(fi, ci)]
    return pf, pc, W
