"""Pins of the oracle's hopping parameter expansion.

* Summed over the 12V unit-vector sources, the HPE-subtracted estimator is
  exact (it equals the dense traces Tr[X (G_u -+ G_d)]) -- the same identity
  that pins the plain estimator, now through Y^4 s and the exact part.
* On lattices with every extent >= 4 the exact diagonal of the first four
  terms is the same at every site and equals the closed form of its two
  non-vanishing orders, written with 4x4 spin matrices (colour gives 3, since
  U U^dag = 1 on the only closed paths, x -> x +- mu -> x):
      3 Tr_s[G A0^-1]
    + 3 kappa^2 sum_mu Tr_s[G (A0^-1 P-_mu A0^-1 P+_mu A0^-1 + A0^-1 P+_mu A0^-1 P-_mu A0^-1)],
  P+-_mu = 1 +- g_mu.
"""
import numpy as np
import pytest

from oracle import dense, dirac, hpe, lattice, tdil
from oracle.gamma import GAMMA, GAMMA5, INSERTIONS
from paper_1401_6750_gb300 import synth


def test_hpe_estimator_exact_over_unit_sources():
    dims = (4, 4, 2, 4)  # small enough for the dense propagators
    kappa, mu = 0.12, 0.07
    u = lattice.effective_links(synth.gauge_links(dims, 0.5, 41), -1)
    g_u, g_d = dense.propagators(u, dims, kappa, mu)
    ex = hpe.exact_ultralocal(hpe.exact_blocks(u, dims, kappa, mu))
    n = g_u.shape[0]
    shp = lattice.shape(dims) + (4, 3)
    # the unit basis plays one noise source: remainders summed over it, the
    # exact part once
    est = hpe.exact_densities(ex)
    eye = np.eye(n, dtype=np.complex128)
    for j0 in range(0, n, 256):
        e = eye[j0:j0 + 256].reshape((-1,) + shp)
        cols = g_u[:, j0:j0 + 256].T.reshape((-1,) + shp)
        est = est + hpe.hpe_densities(u, e, cols, kappa, mu, ultralocal_only=True).sum(axis=1)
    du = dense.exact_densities(g_u, u, dims)
    dd = dense.exact_densities(g_d, u, dims)
    exact = np.concatenate([du - dd, du + dd])
    for g in range(16):
        scale = max(np.max(np.abs(exact[g])), np.max(np.abs(exact[80 + g])))
        for ins in (g, 80 + g):
            assert np.max(np.abs(est[ins] - exact[ins])) <= 1e-11 * scale, ins


@pytest.mark.parametrize("t_bc", [-1, 1])
def test_exact_part_closed_form(t_bc):
    dims = (4, 4, 4, 4)
    kappa, mu = 0.13, 0.05
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 42), t_bc)
    ex = hpe.exact_ultralocal(hpe.exact_blocks(u, dims, kappa, mu))
    mup = 2 * kappa * mu
    one = np.eye(4)
    a0i = (one - 1j * mup * GAMMA5) / (1 + mup * mup)
    inner = a0i.copy()
    for m in range(4):
        pm, pp = one - GAMMA[m], one + GAMMA[m]
        inner = inner + kappa ** 2 * (a0i @ pm @ a0i @ pp @ a0i + a0i @ pp @ a0i @ pm @ a0i)
    for g in range(16):
        want = 3 * np.trace(INSERTIONS[g] @ inner)
        assert np.max(np.abs(ex[g] - want)) < 1e-12, g
    assert np.max(np.abs(hpe.exact_ultralocal_constant(dims, kappa, mu) - ex)) < 1e-12


def test_remainder_suppression():
    """The reason for the subtraction: the remainder field Y^4 s is much
    smaller than s (|Y| ~ 8 kappa / sqrt(1 + mu'^2) per order)."""
    dims = (4, 4, 4, 4)
    kappa, mu = 0.125, 0.01
    u = lattice.effective_links(synth.gauge_links(dims, 0.3, 43), -1)
    s = synth.gaussian_spinor(dims, 44)
    r = hpe.remainder(u, s, kappa, mu)
    assert np.linalg.norm(r) < 1.0 * np.linalg.norm(s)
    assert np.linalg.norm(hpe.remainder(u, s, kappa, mu, order=1)) > 0
