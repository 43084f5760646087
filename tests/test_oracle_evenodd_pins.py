"""Pins of the oracle's even-odd (Schur complement) form of Eq. 1.

Checked against the dense matrix of M (built from the already pinned
``dirac`` operator) with numpy's block algebra, determinant and solver --
none of which use the Schur formulas being tested.
"""
import numpy as np
import pytest

from oracle import dense, dirac, evenodd, lattice, philox
from paper_1401_6750_gb300 import synth

DIMS = (2, 2, 2, 4)


def _setup(dims=DIMS, seed=3):
    return lattice.effective_links(synth.gauge_links(dims, 0.35, seed), -1)


def _index_sets(dims):
    par = evenodd.parity(dims).ravel()
    sites = np.arange(par.size)
    e = (12 * sites[par == 0][:, None] + np.arange(12)).ravel()
    o = (12 * sites[par == 1][:, None] + np.arange(12)).ravel()
    return e, o


def test_parity_checkerboard():
    par = evenodd.parity((4, 2, 2, 2))
    assert par.shape == (2, 2, 2, 4) and par.sum() * 2 == par.size
    # every neighbour, across the periodic wrap too, has the other parity
    for axis in (-1, -2, -3, -4):
        assert np.all(np.roll(par, 1, axis=axis) != par)
    with pytest.raises(ValueError):
        evenodd.parity((4, 3, 2, 2))


@pytest.mark.parametrize("mu", [0.0, 0.07])
def test_block_structure_of_dense_m(mu):
    """Even-even block is the site-local 1 + i mu' g5; hops only couple opposite parities."""
    kappa = 0.13
    u = _setup()
    m = dense.m_matrix(u, DIMS, kappa, mu)
    e, o = _index_sets(DIMS)
    mup = 2 * kappa * mu
    g5 = np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3))
    local = np.kron(np.eye(len(e) // 12), np.eye(12) + 1j * mup * g5)
    assert np.abs(m[np.ix_(e, e)] - local).max() < 1e-14
    assert np.abs(m[np.ix_(o, o)] - local).max() < 1e-14


@pytest.mark.parametrize("mu", [0.01, -0.2])
def test_mhat_is_dense_schur_complement(mu):
    kappa = 0.125
    u = _setup()
    m = dense.m_matrix(u, DIMS, kappa, mu)
    e, o = _index_sets(DIMS)
    want = m[np.ix_(o, o)] - m[np.ix_(o, e)] @ np.linalg.inv(m[np.ix_(e, e)]) @ m[np.ix_(e, o)]
    got = dense.operator_matrix(lambda f: evenodd.apply_mhat(u, f, DIMS, kappa, mu), DIMS)
    gotd = dense.operator_matrix(lambda f: evenodd.apply_mhat_dag(u, f, DIMS, kappa, mu), DIMS)
    assert np.abs(got[np.ix_(o, o)] - want).max() < 1e-13
    assert np.abs(gotd[np.ix_(o, o)] - want.conj().T).max() < 1e-13
    # nothing leaks onto the even sites
    assert np.abs(got[e]).max() == 0.0 and np.abs(gotd[e]).max() == 0.0


def test_determinant_factorises():
    """det M = det M_ee * det Mhat (block LU)."""
    kappa, mu = 0.125, 0.05
    u = _setup(seed=4)
    m = dense.m_matrix(u, DIMS, kappa, mu)
    e, o = _index_sets(DIMS)
    mhat = dense.operator_matrix(lambda f: evenodd.apply_mhat(u, f, DIMS, kappa, mu), DIMS)[np.ix_(o, o)]
    s_full, l_full = np.linalg.slogdet(m)
    s_ee, l_ee = np.linalg.slogdet(m[np.ix_(e, e)])
    s_h, l_h = np.linalg.slogdet(mhat)
    assert abs(l_full - (l_ee + l_h)) < 1e-10
    assert abs(s_full - s_ee * s_h) < 1e-10


def test_schur_solve_matches_dense_solve():
    kappa, mu = 0.125, 0.01
    u = _setup(seed=1)
    eta = philox.z4_source(DIMS, 1001, 0)
    s, iters, res = evenodd.solve(u, eta, DIMS, kappa, mu, rho=1e-13)
    assert res <= 1e-13 and iters > 3
    want = np.linalg.solve(dense.m_matrix(u, DIMS, kappa, mu), eta.ravel()).reshape(eta.shape)
    assert np.linalg.norm((s - want).ravel()) / np.linalg.norm(want.ravel()) < 1e-10
    assert abs(evenodd.normal_residual(u, eta, s, DIMS, kappa, mu) - res) < 1e-12


def test_schur_system_is_better_conditioned():
    """The reason for the form: cond(Mhat^dag Mhat) < cond(M^dag M)."""
    kappa, mu = 0.16, 0.01
    u = _setup(seed=2)
    m = dense.m_matrix(u, DIMS, kappa, mu)
    e, o = _index_sets(DIMS)
    mhat = dense.operator_matrix(lambda f: evenodd.apply_mhat(u, f, DIMS, kappa, mu), DIMS)[np.ix_(o, o)]
    assert np.linalg.cond(mhat) < np.linalg.cond(m)
