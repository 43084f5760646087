"""Derivatives of the one-end loops, for the autograd backward (test only).

The loops of Sec. 2.1.1 are sums over sources of a sesquilinear form of the
solutions, L(mu, eta) = B_mu(s, s) with s = M(mu)^{-1} eta (Eq. 1), and the
tau_3 prefactor -2 i mu' depends on mu explicitly.  Forward mode, plainly:

    ds/dmu = -M^{-1} (dM/dmu) s,       dM/dmu = 2 i kappa g5
    dL/dmu = B(ds, s) + B(s, ds) + B'(s, s)      (B' : prefactor derivative)

and, for a direction d_eta of the sources, ds = M^{-1} d_eta and
dL[d_eta] = B(ds, s) + B(s, ds).  Solves are the oracle's FP64 CG.
"""
import numpy as np

from . import contract, dirac, solver


def loops_and_mu_derivative(u, etas, kappa, mu, dims, moms, rho=1e-12):
    """Sum over the sources of L and dL/dmu, each (160, n_mom, T)."""
    L = 0
    dL = 0
    for eta in etas:
        s, _, _ = solver.solve(u, eta, kappa, mu, rho)
        ds, _, _ = solver.solve(u, -2j * kappa * dirac.gamma5(s), kappa, mu, rho)
        dens = contract.loop_densities_pair(u, s, s, kappa, mu)
        ddens = (contract.loop_densities_pair(u, ds, s, kappa, mu)
                 + contract.loop_densities_pair(u, s, ds, kappa, mu)
                 + contract.loop_densities_pair(u, s, s, kappa, mu, prefactor_derivative=True))
        L = L + contract.project(dens, dims, moms)
        dL = dL + contract.project(ddens, dims, moms)
    return L, dL


def loops_eta_directional(u, etas, detas, kappa, mu, dims, moms, rho=1e-12):
    """Sum over the sources of dL[d_eta] (160, n_mom, T)."""
    dL = 0
    for eta, deta in zip(etas, detas):
        s, _, _ = solver.solve(u, eta, kappa, mu, rho)
        ds, _, _ = solver.solve(u, deta, kappa, mu, rho)
        d = contract.loop_densities_pair(u, ds, s, kappa, mu) + contract.loop_densities_pair(u, s, ds, kappa, mu)
        dL = dL + contract.project(d, dims, moms)
    return dL
