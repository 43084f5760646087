"""Time dilution (Sec. 2.2) on the GPU against the oracle.

* Diluted Z4 sources: bit-exact with ``oracle.tdil.diluted_source``.
* The standard-estimator contraction (both flavours through
  g5-hermiticity, 160 insertions, momentum projection, single-timeslice
  support): against the oracle's literal per-insertion densities on the same
  seeded fields, normwise per insertion: FP64 1e-11, FP32 1e-6 (the
  tolerances of the one-end contraction).
* End to end: the diluted sources of one noise vector solved in FP64 and
  contracted equal the oracle's time-diluted loops to 1e-9.
"""
import numpy as np
import pytest

from gpu_helpers import gauge, round_to, to_device
from oracle import contract, lattice, momenta, tdil
from paper_1401_6750_gb300 import abi, api, synth

pytestmark = pytest.mark.gpu


def _compare(got, want, tol):
    for ins in range(160):
        den = np.linalg.norm(want[ins])
        assert den > 0, ins
        err = np.linalg.norm(got[ins] - want[ins]) / den
        assert err < tol, (ins, err)


@pytest.mark.parametrize("prec", [abi.TSM_F64, abi.TSM_F32, abi.TSM_F16])
def test_diluted_sources_bit_exact(ctx, prec):
    dims = (4, 4, 2, 6)
    g, _ = gauge(ctx, dims, 0.3, 1, -1)
    nat = g.diluted_sources(77, 5, 1, 4, prec)
    got = g.unpack(nat, prec, 4).cpu().numpy()
    for k in range(4):
        assert np.array_equal(got[k], tdil.diluted_source(dims, 77, 5, 1 + k))
    g.close()


@pytest.mark.parametrize("dims,t_bc", [((4, 4, 4, 4), -1), ((6, 4, 2, 8), 1), ((5, 3, 4, 4), -1)])
@pytest.mark.parametrize("prec", [abi.TSM_F64, abi.TSM_F32])
def test_contract_tdil_matches_oracle(ctx, dims, t_bc, prec):
    g, links = gauge(ctx, dims, 0.3, 8, t_bc)
    u = lattice.effective_links(links, t_bc)
    T = dims[3]
    t0 = [0, T - 1, 2, -1]  # three diluted sources and one volume source
    eta = synth.gaussian_spinor(dims, 50, nrhs=4)
    for r, t in enumerate(t0):
        if t >= 0:
            keep = np.zeros(T, dtype=bool)
            keep[t] = True
            eta[r] *= keep[:, None, None, None, None, None]
    eta = round_to(eta, prec)
    s = round_to(synth.gaussian_spinor(dims, 51, nrhs=4), prec)
    moms = momenta.momentum_list(9)
    ne, ns = g.pack(to_device(eta), prec), g.pack(to_device(s), prec)
    got = api.loops_complex(g.contract_tdil(prec, ns, ne, 4, t0, moms))
    want = sum(contract.project(tdil.standard_densities(u, eta[r], s[r]), dims, moms) for r in range(4))
    _compare(got, want, 1e-11 if prec == abi.TSM_F64 else 1e-6)
    # the single-timeslice support is an optimisation only: treating every
    # source as a volume source gives the same loops
    vol = api.loops_complex(g.contract_tdil(prec, ns, ne, 4, None, moms))
    assert np.linalg.norm((vol - got).ravel()) <= 1e-12 * np.linalg.norm(got.ravel()) + 1e-300
    g.close()


def test_tdil_end_to_end_fp64(ctx):
    dims = (4, 4, 4, 4)
    kappa, mu, seed = 0.125, 0.01, 1301
    g, links = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    T = dims[3]
    out = None
    for sid in (0, 1):
        eta = g.diluted_sources(seed, sid, 0, T, abi.TSM_F64)
        sol, st = g.invert(abi.TSM_OP_M, kappa, mu, abi.TSM_SOLVER_F64, 1e-12, eta, T)
        assert all(x["converged"] for x in st)
        out = g.contract_tdil(abi.TSM_F64, sol, eta, T, list(range(T)), moms, out=out, accumulate=out is not None)
    got = api.loops_complex(out) / 2
    want = tdil.tdil_loops(u, dims, kappa, mu, seed, (0, 1), moms)
    _compare(got, want, 1e-9)
    g.close()


def test_tdil_one_sided_momentum_list(ctx):
    """The d flavour is conjugated per site, so a momentum list without -p
    for its p needs nothing else: the loops on {(1, 0, 0), (0, 1, -1)} equal
    the oracle's projection on the same two momenta."""
    dims = (4, 4, 2, 4)
    g, links = gauge(ctx, dims, 0.3, 3, -1, precs=(abi.TSM_F64,))
    u = lattice.effective_links(links, -1)
    eta = synth.gaussian_spinor(dims, 60, nrhs=1)
    s = synth.gaussian_spinor(dims, 61, nrhs=1)
    moms = [(1, 0, 0), (0, 1, -1)]
    ne, ns = g.pack(to_device(eta), abi.TSM_F64), g.pack(to_device(s), abi.TSM_F64)
    got = api.loops_complex(g.contract_tdil(abi.TSM_F64, ns, ne, 1, [-1], moms))
    want = contract.project(tdil.standard_densities(u, eta[0], s[0]), dims, moms)
    _compare(got, want, 1e-11)
    g.close()
