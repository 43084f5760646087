"""One-end-trick contraction and momentum projection (Sec. 2.1.1, Sec. 2.2)
on the GPU against the oracle's literal per-insertion densities.

Both sides receive the same seeded synthetic "solutions" s (Gaussian spinors,
rounded to the storage type for the FP32 path).  The oracle forms every
insertion's density directly and projects with a direct Fourier sum; the GPU
forms the 16 insertion traces per site and projects them separably (x and y
per plane, then z).  Tolerance, normwise per insertion over (momentum,
timeslice): FP64 1e-11; FP32 1e-6 (FP32 products and short x/y sums,
float-float z sums).
"""
import numpy as np
import pytest

from gpu_helpers import gauge, round_to, to_device
from oracle import contract, lattice, momenta
from paper_1401_6750_gb300 import abi, api, synth

pytestmark = pytest.mark.gpu


def _oracle_loops(u, s, kappa, mu, dims, moms):
    acc = 0
    for r in range(s.shape[0]):
        acc = acc + contract.project(contract.loop_densities(u, s[r], kappa, mu), dims, moms)
    return acc


def _compare(got, want, tol):
    worst = 0.0
    for ins in range(160):
        den = np.linalg.norm(want[ins])
        err = np.linalg.norm(got[ins] - want[ins]) / den
        worst = max(worst, err)
        assert err < tol, (ins, err)
    return worst


@pytest.mark.parametrize("dims,t_bc", [((4, 4, 4, 4), -1), ((6, 4, 8, 6), 1), ((5, 3, 4, 4), -1),
                                       ((8, 8, 8, 8), -1)])
@pytest.mark.parametrize("prec", [abi.TSM_F64, abi.TSM_F32])
def test_contraction_matches_oracle(ctx, dims, t_bc, prec):
    kappa, mu = 0.125, 0.01
    g, links = gauge(ctx, dims, 0.3, 4, t_bc)
    u = lattice.effective_links(links, t_bc)
    nsrc = 3
    s = round_to(synth.gaussian_spinor(dims, 40, nrhs=nsrc), prec)
    moms = momenta.momentum_list(9)
    nat = g.pack(to_device(s), prec)
    out = api.loops_complex(g.contract(kappa, mu, prec, nat, nsrc, moms))
    want = _oracle_loops(u, s, kappa, mu, dims, moms)
    _compare(out, want, 1e-11 if prec == abi.TSM_F64 else 1e-6)
    g.close()


@pytest.mark.parametrize("dims,prec,radius", [((40, 32, 2, 2), abi.TSM_F32, 3), ((24, 20, 2, 2), abi.TSM_F64, 8),
                                              ((40, 40, 2, 2), abi.TSM_F64, 8)])
def test_contraction_large_planes(ctx, dims, prec, radius):
    """Planes large enough that the x/y transform takes 4 (FP32, the
    p^2 <= 9 momenta), 2 or a single field (FP64, components up to 8) per
    block instead of 8: its shared memory per block grows with the plane and
    the momentum radius."""
    kappa, mu = 0.125, 0.01
    g, links = gauge(ctx, dims, 0.3, 6, -1)
    u = lattice.effective_links(links, -1)
    s = round_to(synth.gaussian_spinor(dims, 42, nrhs=2), prec)
    if radius == 3:
        moms = momenta.momentum_list(9)
    else:
        moms = [(0, 0, 0), (8, 0, 0), (0, -8, 1), (3, 5, -8), (-7, 2, 4), (1, 1, 1)]
    nat = g.pack(to_device(s), prec)
    out = api.loops_complex(g.contract(kappa, mu, prec, nat, 2, moms))
    want = _oracle_loops(u, s, kappa, mu, dims, moms)
    _compare(out, want, 1e-11 if prec == abi.TSM_F64 else 1e-6)
    g.close()


def test_accumulate_and_momentum_subset(ctx):
    dims = (4, 6, 4, 4)
    kappa, mu = 0.13, 0.02
    g, links = gauge(ctx, dims, 0.3, 5, -1)
    u = lattice.effective_links(links, -1)
    s = synth.gaussian_spinor(dims, 41, nrhs=4)
    moms = [(0, 0, 0), (1, -2, 0), (0, 0, 3)]
    nat = g.pack(to_device(s), abi.TSM_F64)
    field = g.native_bytes(abi.TSM_F64, 1)
    out = g.contract(kappa, mu, abi.TSM_F64, nat[:2 * field], 2, moms)
    out = g.contract(kappa, mu, abi.TSM_F64, nat[2 * field:], 2, moms, out=out, accumulate=True)
    want = _oracle_loops(u, s, kappa, mu, dims, moms)
    _compare(api.loops_complex(out), want, 1e-11)
    g.close()
