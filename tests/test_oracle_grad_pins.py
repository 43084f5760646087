"""Pins of the oracle's loop derivatives (used to check the GPU backward).

* central finite differences of the oracle's own FP64 loops, in mu and in a
  random source direction (solves to 1e-13, step 1e-4: truncation ~1e-8);
* the exact derivative from dense inverses: summed over all 12V unit-vector
  sources the estimator derivative equals Tr[X (dG_u -/+ dG_d)] with
  dG = -G (dM/dmu) G, dM_u/dmu = 2 i kappa g5 = -dM_d/dmu.
"""
import numpy as np

from oracle import contract, dense, dirac, gamma, grad, lattice, momenta, philox
from paper_1401_6750_gb300 import synth

DIMS = (2, 2, 2, 4)


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def test_mu_derivative_matches_finite_difference():
    kappa, mu, h = 0.12, 0.05, 1e-4
    u = lattice.effective_links(synth.gauge_links(DIMS, 0.5, 61), -1)
    moms = momenta.momentum_list(2)
    etas = [philox.z4_source(DIMS, 5, r) for r in range(2)]
    _, dL = grad.loops_and_mu_derivative(u, etas, kappa, mu, DIMS, moms, rho=1e-13)
    lp, _ = grad.loops_and_mu_derivative(u, etas, kappa, mu + h, DIMS, moms, rho=1e-13)
    lm, _ = grad.loops_and_mu_derivative(u, etas, kappa, mu - h, DIMS, moms, rho=1e-13)
    fd = (lp - lm) / (2 * h)
    assert _rel(dL, fd) < 1e-6
    # the explicit tau_3 prefactor term matters: dropping it fails the check
    s = [grad.solver.solve(u, e, kappa, mu, 1e-13)[0] for e in etas]
    expl = sum(contract.project(contract.loop_densities_pair(u, x, x, kappa, mu, True), DIMS, moms) for x in s)
    assert _rel(dL - expl, fd) > 1e-3


def test_eta_direction_matches_finite_difference():
    kappa, mu, h = 0.12, 0.05, 1e-4
    u = lattice.effective_links(synth.gauge_links(DIMS, 0.5, 62), -1)
    moms = momenta.momentum_list(1)
    etas = [philox.z4_source(DIMS, 6, r) for r in range(2)]
    detas = list(synth.gaussian_spinor(DIMS, 63, nrhs=2))
    dL = grad.loops_eta_directional(u, etas, detas, kappa, mu, DIMS, moms, rho=1e-13)
    lp, _ = grad.loops_and_mu_derivative(u, [e + h * d for e, d in zip(etas, detas)], kappa, mu, DIMS, moms, 1e-13)
    lm, _ = grad.loops_and_mu_derivative(u, [e - h * d for e, d in zip(etas, detas)], kappa, mu, DIMS, moms, 1e-13)
    assert _rel(dL, (lp - lm) / (2 * h)) < 1e-6


def test_mu_derivative_exact_from_dense_inverse():
    kappa, mu = 0.12, 0.05
    u = lattice.effective_links(synth.gauge_links(DIMS, 0.5, 64), -1)
    g_u, g_d = dense.propagators(u, DIMS, kappa, mu)
    n = g_u.shape[0]
    g5 = np.kron(np.eye(n // 12), np.kron(gamma.GAMMA5, np.eye(3)))
    dg_u = -g_u @ (2j * kappa * g5) @ g_u
    dg_d = -g_d @ (-2j * kappa * g5) @ g_d
    exact_u = dense.exact_densities(dg_u, u, DIMS)
    exact_d = dense.exact_densities(dg_d, u, DIMS)
    exact = np.concatenate([exact_u - exact_d, exact_u + exact_d])
    shape = (n,) + lattice.shape(DIMS) + (4, 3)
    s = g_u.T.reshape(shape)                           # s_j = G_u e_j
    ds = (-g_u @ (2j * kappa * g5) @ g_u).T.reshape(shape)  # ds_j/dmu
    est = (contract.loop_densities_pair(u, ds, s, kappa, mu) + contract.loop_densities_pair(u, s, ds, kappa, mu)
           + contract.loop_densities_pair(u, s, s, kappa, mu, True)).sum(axis=1)
    assert _rel(est, exact) < 1e-10
