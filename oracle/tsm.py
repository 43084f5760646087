"""Truncated Solver Method (Sec. 2.1).

Sec. 2.1 estimates the loops from ~10^2-10^3 low-precision solves
(rho ~ 1e-2) corrected by ~10-100 high-precision solves (rho ~ 1e-8) and
cites Bali, Collins and Schafer for the method; the estimator is not printed.
Reading (their unbiased form), with disjoint source sets:

    E = (1/N_LP) sum_{r in bulk} L_LP(eta_r)
      + (1/N_HP) sum_{r in corr} [ L_HP(eta_r) - L_LP(eta_r) ]

Source ids: bulk r = 0 .. N_LP-1, correction r = N_LP .. N_LP+N_HP-1, all
drawn with the same noise seed.  The oracle's "LP" and "HP" maps are both its
FP64 CG, stopped at rho_LP and rho_HP.
"""
import numpy as np

from . import contract, philox, solver


def combine(sum_lp_bulk, n_lp, sum_hp, sum_lp_corr, n_hp):
    """TSM estimate from per-source loop SUMS of the three source sets."""
    est = sum_lp_bulk / n_lp
    if n_hp:
        est = est + (sum_hp - sum_lp_corr) / n_hp
    return est


def source_loops(u, dims, kappa, mu, noise_seed, source_id, rho, moms, max_iter=100000):
    """Projected loops of one Z4 source solved to rho: (160, n_mom, T), plus stats."""
    eta = philox.z4_source(dims, noise_seed, source_id)
    s, iters, res = solver.solve(u, eta, kappa, mu, rho, max_iter)
    dens = contract.loop_densities(u, s, kappa, mu)
    return contract.project(dens, dims, moms), iters, res


def tsm_loops(u, dims, kappa, mu, noise_seed, n_lp, n_hp, rho_lp, rho_hp, moms):
    """Full oracle TSM estimate (160, n_mom, T) and the three per-set sums."""
    shape = (contract.N_INSERTIONS, len(moms), dims[3])
    bulk = np.zeros(shape, dtype=np.complex128)
    hp = np.zeros(shape, dtype=np.complex128)
    lpc = np.zeros(shape, dtype=np.complex128)
    for r in range(n_lp):
        bulk += source_loops(u, dims, kappa, mu, noise_seed, r, rho_lp, moms)[0]
    for r in range(n_lp, n_lp + n_hp):
        hp += source_loops(u, dims, kappa, mu, noise_seed, r, rho_hp, moms)[0]
        lpc += source_loops(u, dims, kappa, mu, noise_seed, r, rho_lp, moms)[0]
    return combine(bulk, n_lp, hp, lpc, n_hp), (bulk, hp, lpc)
