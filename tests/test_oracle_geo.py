"""Pins for the oracle's geometry-inclusion local solvers (Section 5.2.3,
oracle/geo.py): the separable fit reproduces separable coefficients exactly;
on a patch with a separable map (x_j depends on eta_j only) the coefficient
diagonal is separable and the off-diagonal entries vanish, so A~_l equals the
true block A_ll, M~_l the true mass and D_A = D_S = 1; on a jittered patch the
scalings restore the true diagonals and P~_A stays SPD; and AF-IETI with these
local solvers reaches the direct solution, in far fewer iterations than the
plain parametric ones on a curved geometry (the paper's reason for the variant)."""
import numpy as np

import afi_workloads as W
from oracle import assembly, geo
from oracle.ieti import AFIETI


def _products(nu, beta):
    d = len(nu)
    def along(v, axis):
        shape = [1] * d
        shape[axis] = len(v)
        return v.reshape(shape)
    diag = []
    for i in range(d):
        t = along(nu[i], i)
        for j in range(d):
            if j != i:
                t = t * along(beta[j], j)
        diag.append(t)
    det = along(beta[0], 0)
    for j in range(1, d):
        det = det * along(beta[j], j)
    return diag, det


def test_separable_fit_is_exact_on_separable_data():
    rng = np.random.default_rng(41)
    for sizes in ((7, 5), (6, 5, 4)):
        nu = [rng.uniform(0.5, 3.0, n) for n in sizes]
        beta = [rng.uniform(0.2, 2.0, n) for n in sizes]
        diag, det = _products(nu, beta)
        fnu, fbeta = geo.separable_fit(diag, det)
        d2, det2 = _products(fnu, fbeta)
        np.testing.assert_allclose(det2, det, rtol=1e-12)
        for a, b in zip(d2, diag):
            np.testing.assert_allclose(a, b, rtol=1e-12)


def _separable_map_problem():
    def geom(e):
        x = e[..., 0] + 0.3 * e[..., 0] ** 2
        y = 0.8 * e[..., 1] + 0.1 * np.sin(np.pi * e[..., 1])
        z = 1.5 * e[..., 2] - 0.2 * e[..., 2] ** 3
        return np.stack([x, y, z], axis=-1)
    return W._structured("separable-map", 3, (2, 1, 1), [[3, 4], [3], [2]], 2, geom)


def test_separable_map_reproduces_the_true_blocks():
    P = _separable_map_problem()
    s = AFIETI(P)
    A = s.assemble()
    for k, g in enumerate(s.geo):
        sl = slice(s.off[k], s.off[k + 1])
        Ak = A[sl][:, sl].tocsr()
        Mk, _ = assembly.mass_block(g)
        lam, mu = P.lame[k]
        gl = geo.GeoLocal(g, lam, mu, s.H[k], Ak, Mk)
        N = s.N[k]
        for l in range(3):
            q = gl.per[l]
            All = Ak[l * N:(l + 1) * N, l * N:(l + 1) * N].toarray()
            At, Mt = q["At"].toarray(), q["Mt"].toarray()
            assert np.abs(At - All).max() <= 1e-10 * np.abs(All).max()
            assert np.abs(Mt - Mk).max() <= 1e-10 * np.abs(Mk).max()
            np.testing.assert_allclose(q["DA"], 1.0, rtol=1e-10)
            np.testing.assert_allclose(q["DS"], 1.0, rtol=1e-10)


def test_scalings_restore_the_true_diagonals_on_a_jittered_patch():
    P = W.config("C2-small")
    s = AFIETI(P)
    A = s.assemble()
    k, g = 0, s.geo[0]
    sl = slice(s.off[k], s.off[k + 1])
    Ak = A[sl][:, sl].tocsr()
    Mk, _ = assembly.mass_block(g)
    lam, mu = P.lame[k]
    gl = geo.GeoLocal(g, lam, mu, s.H[k], Ak, Mk)
    N = s.N[k]
    for l in range(3):
        q = gl.per[l]
        All = Ak[l * N:(l + 1) * N, l * N:(l + 1) * N]
        Pd = (q["At"] + q["Mt"] / s.H[k] ** 2).toarray()
        Ps = np.sqrt(q["DA"])[:, None] * Pd * np.sqrt(q["DA"])[None, :]
        np.testing.assert_allclose(np.diag(Ps), All.diagonal() + np.diag(Mk) / s.H[k] ** 2, rtol=1e-12)
        assert np.linalg.eigvalsh(0.5 * (Ps + Ps.T)).min() > 0.0
        np.testing.assert_allclose(q["DS"] * q["At"].diagonal(), All.diagonal(), rtol=1e-12)
        # P~_A^{-1} inverts the scaled matrix
        r = np.random.default_rng(l).standard_normal(N)
        np.testing.assert_allclose(Ps @ gl.PA_inv(l, r), r, rtol=1e-9, atol=1e-11 * np.abs(r).max())


def test_geo_solve_on_a_curved_geometry():
    P = W.quarter_annulus(grid=(2, 2, 1), p=2, nel=4, name="annulus-tiny")
    sg, si = AFIETI(P, precond="geo"), AFIETI(P)
    f = sg.load(W.body_force_coeffs(P))
    u, lam, info = sg.solve(f, tol=1e-10)
    _, _, info_i = si.solve(f, tol=1e-10)
    ud, ld = sg.direct_solve(f)
    assert np.linalg.norm(u - ud) <= 1e-7 * np.linalg.norm(ud)
    assert np.linalg.norm(lam - ld) <= 1e-7 * np.linalg.norm(ld)
    assert info["iters"] < 0.6 * info_i["iters"]
