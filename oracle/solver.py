"""Conjugate gradient for Eq. 1, M s = eta, through the normal equations.

The paper (Sec. 2) hands Eq. 1 to QUDA's twisted-mass CG inverter; the CG it
runs is on the Hermitian positive-definite M^dag M.  Textbook CG (Hestenes and
Stiefel) in FP64:

    b = M^dag eta,  x_0 = 0,  r_0 = b,  p_0 = r_0
    alpha_k = (r_k, r_k) / (p_k, M^dag M p_k)
    x_{k+1} = x_k + alpha_k p_k
    r_{k+1} = r_k - alpha_k M^dag M p_k
    beta_k  = (r_{k+1}, r_{k+1}) / (r_k, r_k)
    p_{k+1} = r_{k+1} + beta_k p_k

Stopping rule (the residual rho of Sec. 2.1 is not defined in the paper; this
is the reading used throughout): iterate while |r_k| > rho |b|; on exit
recompute the true residual b - M^dag M x.  If it is still above rho |b| the
iteration restarts from r = b - M^dag M x, p = r.  ``max_iter`` bounds the
total number of iterations.
"""
import numpy as np

from . import dirac


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def norm2(a):
    return float(np.vdot(a.ravel(), a.ravel()).real)


def cg_normal(u, b, kappa, mu, rho, max_iter, x0=None):
    """Solve (M^dag M) x = b.  Returns (x, iterations, true relative residual)."""
    return cg(lambda v: dirac.apply_MdagM(u, v, kappa, mu), b, rho, max_iter, x0)


def cg(apply, b, rho, max_iter, x0=None):
    """The CG above for any Hermitian positive-definite map ``apply``."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bb = norm2(b)
    if bb == 0.0:
        return x, 0, 0.0
    r = b - apply(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = norm2(r)
    it = 0
    while True:
        while rr > rho * rho * bb and it < max_iter:
            ap = apply(p)
            alpha = rr / vdot(p, ap).real
            x = x + alpha * p
            r = r - alpha * ap
            rr_new = norm2(r)
            p = r + (rr_new / rr) * p
            rr = rr_new
            it += 1
        r = b - apply(x)
        rr = norm2(r)
        if rr <= rho * rho * bb or it >= max_iter:
            return x, it, float(np.sqrt(rr / bb))
        p = r.copy()


def solve(u, eta, kappa, mu, rho, max_iter=100000):
    """s = M^{-1} eta via CG on M^dag M x = M^dag eta (Eq. 1)."""
    b = dirac.apply_Mdag(u, eta, kappa, mu)
    return cg_normal(u, b, kappa, mu, rho, max_iter)
