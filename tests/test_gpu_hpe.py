"""Hopping parameter expansion (HPE) of the standard estimator on the GPU
against the oracle.

* The HPE contraction on the same seeded fields (diluted and volume
  sources, both boundary conditions) against ``oracle.hpe.hpe_densities``
  projected: normwise per insertion FP64 1e-10, FP32 1e-5 (four FP32 hops
  with reconstructed links before the contraction).
* End to end: the time-diluted FP64 solves of one noise vector with HPE
  against the oracle's sum over timeslices, 1e-9.
* Lattices with an extent below 4 are refused.
"""
import numpy as np
import pytest

from gpu_helpers import gauge, round_to, to_device
from oracle import contract, hpe, lattice, momenta, tdil
from paper_1401_6750_gb300 import abi, api, synth

pytestmark = pytest.mark.gpu


def _compare(got, want, tol):
    for ins in range(160):
        den = np.linalg.norm(want[ins])
        assert den > 0, ins
        err = np.linalg.norm(got[ins] - want[ins]) / den
        assert err < tol, (ins, err)


@pytest.mark.parametrize("dims,t_bc", [((4, 4, 4, 4), -1), ((6, 4, 4, 8), 1)])
@pytest.mark.parametrize("prec", [abi.TSM_F64, abi.TSM_F32])
def test_hpe_contract_matches_oracle(ctx, dims, t_bc, prec):
    kappa, mu = 0.13, 0.04
    g, links = gauge(ctx, dims, 0.3, 9, t_bc)
    u = lattice.effective_links(links, t_bc)
    T = dims[3]
    t0 = [1, T - 1, -1]
    eta = synth.gaussian_spinor(dims, 60, nrhs=3)
    for r, t in enumerate(t0):
        if t >= 0:
            keep = np.zeros(T, dtype=bool)
            keep[t] = True
            eta[r] *= keep[:, None, None, None, None, None]
    eta = round_to(eta, prec)
    s = round_to(synth.gaussian_spinor(dims, 61, nrhs=3), prec)
    moms = momenta.momentum_list(9)
    got = api.loops_complex(g.contract_hpe(kappa, mu, prec, g.pack(to_device(s), prec), g.pack(to_device(eta), prec),
                                           3, t0, moms))
    ex = hpe.exact_ultralocal_constant(dims, kappa, mu)
    want = 0
    for r, t in enumerate(t0):
        d = hpe.hpe_densities(u, eta[r], s[r], kappa, mu, ex, support=None if t < 0 else [t])
        want = want + contract.project(d, dims, moms)
    _compare(got, want, 1e-10 if prec == abi.TSM_F64 else 1e-5)
    g.close()


def test_hpe_time_diluted_end_to_end_fp64(ctx):
    dims = (4, 4, 4, 4)
    kappa, mu, seed = 0.125, 0.01, 1401
    g, links = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    T = dims[3]
    eta = g.diluted_sources(seed, 0, 0, T, abi.TSM_F64)
    sol, st = g.invert(abi.TSM_OP_M, kappa, mu, abi.TSM_SOLVER_F64, 1e-12, eta, T)
    got = api.loops_complex(g.contract_hpe(kappa, mu, abi.TSM_F64, sol, eta, T, list(range(T)), moms))
    ex = hpe.exact_ultralocal_constant(dims, kappa, mu)
    from oracle import solver
    want = 0
    for t0 in range(T):
        e = tdil.diluted_source(dims, seed, 0, t0)
        s, _, _ = solver.solve(u, e, kappa, mu, 1e-12)
        want = want + contract.project(hpe.hpe_densities(u, e, s, kappa, mu, ex, support=[t0]), dims, moms)
    _compare(got, want, 1e-9)
    g.close()


def test_hpe_rejects_short_extents(ctx):
    dims = (4, 4, 2, 4)
    g, _ = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    eta = g.diluted_sources(1, 0, 0, 1, abi.TSM_F64)
    with pytest.raises(abi.TsmError):
        g.contract_hpe(0.125, 0.01, abi.TSM_F64, eta, eta, 1, [0], momenta.momentum_list(1))
    g.close()
