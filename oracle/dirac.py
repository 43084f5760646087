"""Twisted-mass Wilson operator (the matrix M of Eq. 1).

The paper solves M s = eta (Eq. 1) with QUDA's twisted-mass operator but
prints no formula for M.  The oracle uses the standard kappa-normalised form
(u flavour, twisted basis):

    M(mu) = A + i mu' gamma_5,        mu' = 2 kappa mu
    A psi(x) = psi(x) - kappa sum_mu [ (1 - gamma_mu) U_mu(x)          psi(x+mu)
                                     + (1 + gamma_mu) U_mu(x-mu)^dag   psi(x-mu) ]

and its adjoint, written out term by term (no gamma_5 trick):

    M^dag(mu) = A^dag - i mu' gamma_5
    A^dag psi(x) = psi(x) - kappa sum_mu [ (1 + gamma_mu) U_mu(x)        psi(x+mu)
                                         + (1 - gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]

``u`` is the array of effective links (boundary sign already applied, see
``lattice.effective_links``); spinors have shape (t, z, y, x, 4, 3).
"""
import numpy as np

from . import lattice
from .gamma import GAMMA, GAMMA5


def colour_mul(u, psi):
    """(U psi)_{s a} = sum_b U_{a b} psi_{s b} for every site and spin s."""
    return np.matmul(psi, np.swapaxes(u, -1, -2))


def colour_mul_dag(u, psi):
    """(U^dag psi)_{s a} = sum_b conj(U_{b a}) psi_{s b}."""
    return np.matmul(psi, np.conj(u))


def spin_mul(g, psi):
    """(G psi)_{s a} = sum_r G_{s r} psi_{r a}."""
    return np.matmul(g, psi)


def hop(u, psi, sign):
    """sum_mu [(1 + sign*g_mu) U_mu(x) psi(x+mu) + (1 - sign*g_mu) U_mu(x-mu)^dag psi(x-mu)].

    sign = -1 gives the hopping term of A, sign = +1 that of A^dag.
    """
    out = np.zeros_like(psi)
    for mu in range(4):
        f = colour_mul(u[..., mu, :, :], lattice.fwd(psi, mu))
        b = colour_mul_dag(lattice.bwd(u[..., mu, :, :], mu), lattice.bwd(psi, mu))
        out += f + sign * spin_mul(GAMMA[mu], f)
        out += b - sign * spin_mul(GAMMA[mu], b)
    return out


def apply_A(u, psi, kappa):
    """Wilson part A (twisted mass zero)."""
    return psi - kappa * hop(u, psi, -1.0)


def apply_Adag(u, psi, kappa):
    return psi - kappa * hop(u, psi, +1.0)


def apply_M(u, psi, kappa, mu):
    return apply_A(u, psi, kappa) + 1j * (2.0 * kappa * mu) * spin_mul(GAMMA5, psi)


def apply_Mdag(u, psi, kappa, mu):
    return apply_Adag(u, psi, kappa) - 1j * (2.0 * kappa * mu) * spin_mul(GAMMA5, psi)


def apply_MdagM(u, psi, kappa, mu):
    return apply_Mdag(u, apply_M(u, psi, kappa, mu), kappa, mu)


def gamma5(psi):
    return spin_mul(GAMMA5, psi)
