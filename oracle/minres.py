"""Preconditioned MINRES (Paige & Saunders 1975), written out as the textbook
Lanczos recurrence with Givens rotations; the solver used by AF-IETI
(Section 4, zero initial guess, relative tolerance on the preconditioned
residual estimate).  Oracle code: test infrastructure only."""
from __future__ import annotations

import math

import numpy as np


def next_true_check(itn, true_rel, tol, hist):
    """Iteration of the next true-residual check after a failed one at `itn`:
    extrapolate the estimate's mean reduction per iteration over the last five
    iterations, q = (hist[itn] / hist[itn-5])^(1/5), to the number of
    iterations that would reduce true_rel to tol; at least 5, at most 50."""
    extra = 5
    if itn >= 5 and hist[itn - 5] > 0 and hist[itn] > 0:
        q = (hist[itn] / hist[itn - 5]) ** 0.2
        if 0.0 < q < 1.0:
            extra = math.ceil(math.log(true_rel / tol) / (-math.log(q)))
    return itn + min(max(extra, 5), 50)


def minres(Aop, b, Mop=None, tol=1e-8, maxit=1000, callback=None, true_check=None):
    """Solve A x = b for symmetric A with SPD preconditioner M^{-1} = Mop.

    Stops when the recurrence estimate phibar/beta1 of the preconditioned
    residual falls to tol; if ``true_check(x)`` is given (the true relative
    residual ||b - A x|| / ||b||), iterations continue past that point until
    the true residual is also at or below tol, re-checked at the iteration
    given by next_true_check.  Returns (x, info) with info = {iters,
    relres_est, history}."""
    Mop = Mop or (lambda v: v)
    n = b.shape[0]
    x = np.zeros(n)
    r1 = b.copy()
    y = Mop(r1)
    beta1 = float(np.dot(r1, y))
    if beta1 < 0:
        raise ArithmeticError("preconditioner is not positive definite")
    beta1 = np.sqrt(beta1)
    if beta1 == 0.0:
        return x, {"iters": 0, "relres_est": 0.0, "history": [0.0]}
    oldb, beta = 0.0, beta1
    dbar, epsln, phibar = 0.0, 0.0, beta1
    cs, sn = -1.0, 0.0
    w = np.zeros(n)
    w2 = np.zeros(n)
    r2 = r1.copy()
    hist = [1.0]
    itn = 0
    next_check = 0
    while itn < maxit:
        itn += 1
        s = 1.0 / beta
        v = s * y
        y = Aop(v)
        if itn >= 2:
            y = y - (beta / oldb) * r1
        alfa = float(np.dot(v, y))
        y = y - (alfa / beta) * r2
        r1 = r2
        r2 = y
        y = Mop(r2)
        oldb = beta
        beta2 = float(np.dot(r2, y))
        if beta2 < 0:
            raise ArithmeticError("preconditioner is not positive definite")
        beta = np.sqrt(beta2)
        oldeps = epsln
        delta = cs * dbar + sn * alfa
        gbar = sn * dbar - cs * alfa
        epsln = sn * beta
        dbar = -cs * beta
        gamma = max(np.hypot(gbar, beta), np.finfo(float).tiny)
        cs = gbar / gamma
        sn = beta / gamma
        phi = cs * phibar
        phibar = sn * phibar
        w1 = w2
        w2 = w
        w = (v - oldeps * w1 - delta * w2) / gamma
        x = x + phi * w
        rel = phibar / beta1
        hist.append(rel)
        if callback is not None:
            callback(itn, x, rel)
        if rel <= tol:
            if true_check is None:
                break
            if itn >= next_check:
                tr = true_check(x)
                if tr <= tol:
                    break
                next_check = next_true_check(itn, tr, tol, hist)
    return x, {"iters": itn, "relres_est": float(phibar / beta1), "history": hist}
