"""Pins of the oracle's time-diluted sources and standard estimator.

The estimator is pinned by the identity that fixes every term of it: summed
over the 12V unit-vector sources (each lives on one timeslice, so the sum is
also a complete time dilution), eta(y)^dag K s(z) gives Tr[K G_u(z, y)]
exactly and the g5-hermiticity route gives Tr[K G_d(z, y)] exactly; both are
compared with the dense propagators of the already pinned operator.
"""
import numpy as np
import pytest

from oracle import dense, lattice, philox, tdil
from paper_1401_6750_gb300 import synth

DIMS = (2, 2, 2, 4)


def test_diluted_sources_partition_the_volume_source():
    dims = (2, 4, 2, 6)
    eta = philox.z4_source(dims, 77, 5)
    parts = [tdil.diluted_source(dims, 77, 5, t0) for t0 in range(dims[3])]
    assert np.array_equal(sum(parts), eta)
    for t0, p in enumerate(parts):
        others = np.delete(p, t0, axis=0)
        assert np.all(others == 0) and np.array_equal(p[t0], eta[t0])


@pytest.mark.parametrize("t_bc", [-1, 1])
def test_standard_estimator_exact_over_unit_sources(t_bc):
    kappa, mu = 0.12, 0.05
    u = lattice.effective_links(synth.gauge_links(DIMS, 0.5, 31), t_bc)
    g_u, g_d = dense.propagators(u, DIMS, kappa, mu)
    n = g_u.shape[0]
    shp = lattice.shape(DIMS) + (4, 3)
    est = 0
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        est = est + tdil.standard_densities(u, e.reshape(shp), g_u[:, j].reshape(shp))
    du = dense.exact_densities(g_u, u, DIMS)
    dd = dense.exact_densities(g_d, u, DIMS)
    exact = np.concatenate([du - dd, du + dd])
    for ins in range(160):
        scale = max(np.max(np.abs(exact[ins])), 1e-12)
        assert np.max(np.abs(est[ins] - exact[ins])) <= 1e-10 * scale, ins


def test_d_flavour_route_is_not_the_u_route():
    """A slip that reused the u estimator for d would make u - d vanish; the
    tau_3 combination is non-zero for mu != 0."""
    kappa, mu = 0.12, 0.05
    u = lattice.effective_links(synth.gauge_links(DIMS, 0.5, 32), -1)
    eta = tdil.diluted_source(DIMS, 3, 0, 1)
    from oracle import solver
    s, _, _ = solver.solve(u, eta, kappa, mu, 1e-13)
    d = tdil.standard_densities(u, eta, s)
    assert np.max(np.abs(d[0:16])) > 1e-3
    # ultra-local densities vanish off the source's timeslice
    assert np.max(np.abs(np.delete(d[0:16], 1, axis=1))) == 0.0


def test_standard_density_subset_equals_full():
    """standard_densities(only=...) evaluates the same formulas for the listed
    insertions (both flavour combinations) and leaves the rest zero."""
    import numpy as np
    from oracle import lattice, tdil
    from paper_1401_6750_gb300 import synth
    dims = (2, 2, 2, 4)
    u = lattice.effective_links(synth.gauge_links(dims, 0.4, 71), -1)
    eta = tdil.diluted_source(dims, 72, 0, 1)
    s = synth.gaussian_spinor(dims, 73)
    full = tdil.standard_densities(u, eta, s)
    part = tdil.standard_densities(u, eta, s, only={15, 17, 152})
    keep = {15, 95, 17, 97, 72, 152}
    for i in range(160):
        if i in keep:
            assert np.array_equal(part[i], full[i])
        else:
            assert not np.any(part[i])
