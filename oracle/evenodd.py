"""Even-odd (Schur complement) form of Eq. 1.  TEST INFRASTRUCTURE ONLY.

Sites split by parity (x + y + z + t even or odd).  The hopping term of M only
connects sites of opposite parity, so in that ordering

    M = [[M_ee, M_eo], [M_oe, M_oo]],   M_ee = M_oo = 1 + i mu' g5 (site-local),
    M_eo = -kappa H_eo,  M_oe = -kappa H_oe      (H = dirac.hop(u, ., -1))

and M s = eta is equivalent to

    Mhat s_o = eta_o - M_oe M_ee^{-1} eta_e,    Mhat = M_oo - M_oe M_ee^{-1} M_eo
    s_e = M_ee^{-1} (eta_e - M_eo s_o),         M_ee^{-1} = (1 - i mu' g5) / (1 + mu'^2).

The paper (Sec. 2) solves Eq. 1 with QUDA's twisted-mass CG and does not say
whether it preconditions; the solution of Eq. 1 is the same either way.  The
odd-site system is solved here by the textbook CG on Mhat^dag Mhat (same
stopping rule as ``solver``, applied to b = Mhat^dag eta_hat).  Fields keep the
full lattice shape and are zero on the sites of the other parity.
"""
import numpy as np

from . import dirac, lattice, solver


def parity(dims):
    """(t, z, y, x) integer array: 0 on even sites, 1 on odd sites.  The split
    is a checkerboard of the hopping term only when every extent is even."""
    if any(n % 2 for n in dims):
        raise ValueError("the even-odd form needs even extents, got %s" % (dims,))
    x, y, z, t = lattice.coords(dims)
    return (x + y + z + t) & 1


def restrict(psi, dims, p):
    """psi on the sites of parity p, zero elsewhere."""
    return psi * (parity(dims) == p)[..., None, None]


def diag_inv(psi, kappa, mu):
    """M_ee^{-1} psi = (1 - i mu' g5) psi / (1 + mu'^2), mu' = 2 kappa mu."""
    mup = 2.0 * kappa * mu
    return (psi - 1j * mup * dirac.gamma5(psi)) / (1.0 + mup * mup)


def apply_mhat(u, v, dims, kappa, mu):
    """Mhat v for v on the odd sites: (1 + i mu' g5) v - kappa^2 H_oe M_ee^{-1} H_eo v."""
    mup = 2.0 * kappa * mu
    v = restrict(v, dims, 1)
    w = restrict(dirac.hop(u, v, -1.0), dims, 0)
    w = diag_inv(w, kappa, mu)
    hw = restrict(dirac.hop(u, w, -1.0), dims, 1)
    return v + 1j * mup * dirac.gamma5(v) - kappa * kappa * hw


def apply_mhat_dag(u, v, dims, kappa, mu):
    """Mhat^dag v, written out term by term: H^dag is the hop with sign +1 and
    (M_ee^{-1})^dag = (1 + i mu' g5) / (1 + mu'^2)."""
    mup = 2.0 * kappa * mu
    v = restrict(v, dims, 1)
    w = restrict(dirac.hop(u, v, +1.0), dims, 0)
    w = (w + 1j * mup * dirac.gamma5(w)) / (1.0 + mup * mup)
    hw = restrict(dirac.hop(u, w, +1.0), dims, 1)
    return v - 1j * mup * dirac.gamma5(v) - kappa * kappa * hw


def schur_source(u, eta, dims, kappa, mu):
    """eta_hat = eta_o - M_oe M_ee^{-1} eta_e = eta_o + kappa H_oe M_ee^{-1} eta_e."""
    ye = diag_inv(restrict(eta, dims, 0), kappa, mu)
    return restrict(eta, dims, 1) + kappa * restrict(dirac.hop(u, ye, -1.0), dims, 1)


def reconstruct(u, eta, s_o, dims, kappa, mu):
    """Full solution: s_o on odd sites, s_e = M_ee^{-1}(eta_e + kappa H_eo s_o) on even sites."""
    s_o = restrict(s_o, dims, 1)
    rhs = restrict(eta, dims, 0) + kappa * restrict(dirac.hop(u, s_o, -1.0), dims, 0)
    return diag_inv(rhs, kappa, mu) + s_o


def normal_residual(u, eta, s, dims, kappa, mu):
    """|b - Mhat^dag Mhat s_o| / |b| with b = Mhat^dag eta_hat (the quantity rho bounds)."""
    b = apply_mhat_dag(u, schur_source(u, eta, dims, kappa, mu), dims, kappa, mu)
    s_o = restrict(s, dims, 1)
    r = b - apply_mhat_dag(u, apply_mhat(u, s_o, dims, kappa, mu), dims, kappa, mu)
    return float(np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel()))


def solve(u, eta, dims, kappa, mu, rho, max_iter=100000):
    """s = M^{-1} eta through the odd-site Schur system.  Returns (s, iterations,
    true relative residual of the odd-site normal equations)."""
    b = apply_mhat_dag(u, schur_source(u, eta, dims, kappa, mu), dims, kappa, mu)
    normal = lambda v: apply_mhat_dag(u, apply_mhat(u, v, dims, kappa, mu), dims, kappa, mu)
    s_o, iters, res = solver.cg(normal, b, rho, max_iter)
    return reconstruct(u, eta, s_o, dims, kappa, mu), iters, res
