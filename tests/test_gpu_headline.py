"""The headline configuration, 24^3 x 48 (eps 0.25, gauge seed 3,
kappa 0.125, mu 0.005, noise seed 1003), checked against the oracle at full
size rather than trusted from small lattices:

* even-odd FP16 LP solves (the bulk of the TSM): the odd-site normal
  residual of each returned vector, recomputed by the oracle in FP64, is at
  most rho_LP = 1e-2;
* an even-odd HP solve (FP32 CG, float-float reliable updates): recomputed
  residual at most rho_HP = 1e-8;
* the FP32 contraction of that HP solution against the oracle's FP64
  densities and direct Fourier sums for a subset of insertions (scalar and
  g5 of both flavour structures, two derivative insertions), all 123
  momenta, every timeslice: 1e-6 normwise per insertion;
* the standard-estimator contraction likewise;
* the bench's TSM step itself: its LP-correction and HP sums against the
  oracle's contraction of the regenerated correction vectors, and its
  combination.
"""
import numpy as np
import pytest

from gpu_helpers import gauge
from oracle import contract, evenodd, lattice, momenta, philox
from paper_1401_6750_gb300 import abi, api

pytestmark = pytest.mark.gpu
EO = abi.TSM_SOLVER_EO
DIMS = (24, 24, 24, 48)
KAPPA, MU, SEED = 0.125, 0.005, 1003


@pytest.fixture(scope="module")
def headline(ctx):
    g, links = gauge(ctx, DIMS, 0.25, 3, -1, precs=(abi.TSM_F64, abi.TSM_F32, abi.TSM_F16))
    yield g, lattice.effective_links(links, -1)
    g.close()


def test_headline_lp_solves_meet_rho(headline):
    g, u = headline
    n = 2
    nat, st = g.solve_sources(KAPPA, MU, abi.TSM_SOLVER_LP_F16 | EO, 1e-2, SEED, 0, n, nrhs_per_launch=n)
    x = g.unpack(nat, abi.TSM_F32, n).cpu().numpy()
    for k in range(n):
        res = evenodd.normal_residual(u, philox.z4_source(DIMS, SEED, k), x[k], DIMS, KAPPA, MU)
        assert st[k]["converged"] == 1 and res <= 1e-2, (k, res, st[k])


def test_headline_hp_solve_and_contraction(headline):
    g, u = headline
    src = 32  # the first correction source of a 32 + 2 source step
    nat, st = g.solve_sources(KAPPA, MU, abi.TSM_SOLVER_F32_RELIABLE | EO, 1e-8, SEED, src, 1)
    x = g.unpack(nat, abi.TSM_F64, 1).cpu().numpy()[0]
    res = evenodd.normal_residual(u, philox.z4_source(DIMS, SEED, src), x, DIMS, KAPPA, MU)
    assert st[0]["converged"] == 1 and res <= 1e-8, (res, st[0])
    # the driver contracts HP solutions in FP32
    s32 = g.pack(g.unpack(nat, abi.TSM_F64, 1), abi.TSM_F32)
    moms = momenta.momentum_list(9)
    got = api.loops_complex(g.contract(KAPPA, MU, abi.TSM_F32, s32, 1, moms))
    xs = g.unpack(s32, abi.TSM_F32, 1).cpu().numpy()[0]
    sel = [0, 15, 80, 95,
           contract.insertion_index(0, True, 0, 1), contract.insertion_index(1, True, 3, 8)]
    dens = contract.loop_densities(u, xs, KAPPA, MU, only=set(sel))
    want = contract.project(dens[sel], DIMS, moms)
    for k, ins in enumerate(sel):
        err = np.linalg.norm(got[ins] - want[k]) / np.linalg.norm(want[k])
        assert err < 1e-6, (ins, err)


@pytest.mark.parametrize("t0", [5, -1])
def test_headline_standard_estimator_contraction(headline, t0):
    """The standard-estimator contraction (time dilution: the source kept on
    timeslice 5; and a volume source) of an HP solution in FP32 against the
    oracle's FP64 densities and direct Fourier sums, the same six insertions,
    all 123 momenta: 1e-6."""
    from oracle import tdil
    g, u = headline
    moms = momenta.momentum_list(9)
    if t0 >= 0:
        eta_nat = g.diluted_sources(SEED, 40, t0, 1, abi.TSM_F64)
    else:
        eta_nat = g.sources(SEED, 40, 1, abi.TSM_F64)
    sol, st = g.invert(abi.TSM_OP_M, KAPPA, MU, abi.TSM_SOLVER_F32_RELIABLE | EO, 1e-9, eta_nat, 1)
    s32 = g.pack(g.unpack(sol, abi.TSM_F64, 1), abi.TSM_F32)
    e32 = g.pack(g.unpack(eta_nat, abi.TSM_F64, 1), abi.TSM_F32)
    got = api.loops_complex(g.contract_tdil(abi.TSM_F32, s32, e32, 1, [t0], moms))
    xs = g.unpack(s32, abi.TSM_F32, 1).cpu().numpy()[0]
    eta = g.unpack(eta_nat, abi.TSM_F64, 1).cpu().numpy()[0]
    sel = [0, 15, 80, 95,
           contract.insertion_index(0, True, 0, 1), contract.insertion_index(1, True, 3, 8)]
    dens = tdil.standard_densities(u, eta, xs, only=set(sel))
    want = contract.project(dens[sel], DIMS, moms)
    for k, ins in enumerate(sel):
        err = np.linalg.norm(got[ins] - want[k]) / np.linalg.norm(want[k])
        assert err < 1e-6, (t0, ins, err)


def test_headline_tsm_step_correction_sums(headline):
    """The bench's TSM step itself (32 FP16 LP + 2 HP sources, 32 right-hand
    sides per launch, even-odd maps, the correction chain on its own stream):
    the driver's LP-correction and HP sums equal the oracle's FP64 contraction
    of the two correction sources' LP and HP vectors, regenerated source by
    source (one map per source, whatever the batch), on the six insertions
    above and all 123 momenta (1e-6); the estimate is the combination of the
    driver's three sums."""
    g, u = headline
    moms = momenta.momentum_list(9)
    lp, hp = abi.TSM_SOLVER_LP_F16 | EO, abi.TSM_SOLVER_F32_RELIABLE | EO
    n_lp, n_hp = 32, 2
    est, parts, st = g.tsm(KAPPA, MU, n_lp, n_hp, 1e-2, 1e-8, lp, hp, SEED, moms, nrhs_per_launch=32,
                           want_parts=True)
    assert st["n_not_converged"] == 0
    comb = parts[0] / n_lp + (parts[1] - parts[2]) / n_hp
    assert np.abs(est - comb).max() <= 1e-12 * np.abs(est).max()
    lp_nat, _ = g.solve_sources(KAPPA, MU, lp, 1e-2, SEED, n_lp, n_hp, nrhs_per_launch=32)
    hp_nat, _ = g.solve_sources(KAPPA, MU, hp, 1e-8, SEED, n_lp, n_hp, nrhs_per_launch=32)
    x_lp = g.unpack(lp_nat, abi.TSM_F32, n_hp).cpu().numpy()
    # the driver contracts HP solutions in FP32
    x_hp = g.unpack(g.pack(g.unpack(hp_nat, abi.TSM_F64, n_hp), abi.TSM_F32), abi.TSM_F32, n_hp).cpu().numpy()
    sel = [0, 15, 80, 95,
           contract.insertion_index(0, True, 0, 1), contract.insertion_index(1, True, 3, 8)]
    for which, x in ((2, x_lp), (1, x_hp)):
        want = sum(contract.project(contract.loop_densities(u, x[r], KAPPA, MU, only=set(sel))[sel], DIMS, moms)
                   for r in range(n_hp))
        for k, ins in enumerate(sel):
            err = np.linalg.norm(parts[which][ins] - want[k]) / np.linalg.norm(want[k])
            assert err < 1e-6, (which, ins, err)
