"""The headline truncated-solver estimate with the 16-bit LP map against the
oracle, on identical sources (Sec. 2.1).

A truncated solve is not unique (it depends on the iteration path), so the
oracle cannot reproduce the LP solution vectors themselves.  What is unique,
and checked here, is the contraction and combination of the vectors the
library produced:

* the LP map is a deterministic function of each source (per right-hand
  side arithmetic that does not depend on its batch mates), so
  tsm_solve_sources with the same solver, rho and source ids regenerates the
  very vectors the TSM driver contracted -- the library's own contraction of
  them reproduces the driver's per-set sums;
* the oracle's FP64 contraction of those downloaded vectors matches the
  driver's bulk sum and LP-correction sum, the HP sum matches the oracle's
  converged solves, and the combined estimate matches the oracle's
  combination of the three -- each within 1e-6 normwise per insertion;
* every downloaded LP vector has an oracle-recomputed true residual <= rho;
* separately, the estimate is statistically consistent with the exact
  traces of a dense inverse (a crude LP map, so that the LP-only mean is
  visibly biased while the corrected one is not).
"""
import numpy as np
import pytest

from gpu_helpers import gauge
from oracle import contract, dense, evenodd, lattice, momenta, philox, solver, tsm
from paper_1401_6750_gb300 import abi, api

pytestmark = pytest.mark.gpu
EO = abi.TSM_SOLVER_EO
TOL = 1e-6  # FP32 solves and contraction against the FP64 oracle


def _rel(got, want):
    return max(np.linalg.norm(got[i] - want[i]) / np.linalg.norm(want[i]) for i in range(want.shape[0]))


def _normal_residual(u, eta, x, dims, kappa, mu, eo):
    if eo:
        return evenodd.normal_residual(u, eta, x, dims, kappa, mu)
    b = solver.dirac.apply_Mdag(u, eta, kappa, mu)
    r = b - solver.dirac.apply_MdagM(u, x, kappa, mu)
    return np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("lp_solver", [abi.TSM_SOLVER_LP_F16 | EO, abi.TSM_SOLVER_LP_BF16 | EO,
                                       abi.TSM_SOLVER_LP_F16])
def test_tsm_lowprec_sums_match_oracle_contraction(ctx, lp_solver):
    dims = (6, 4, 4, 8)
    kappa, mu, seed = 0.125, 0.01, 1302
    rho_lp, rho_hp = 1e-2, 1e-8
    hp_solver = abi.TSM_SOLVER_F32_RELIABLE | (lp_solver & EO)
    g, links = gauge(ctx, dims, 0.3, 2, -1)
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    n_lp, n_hp, nb = 8, 3, 4
    est, parts, st = g.tsm(kappa, mu, n_lp, n_hp, rho_lp, rho_hp, lp_solver, hp_solver, seed, moms,
                           nrhs_per_launch=nb, want_parts=True)
    assert st["n_not_converged"] == 0
    # the LP vectors the driver contracted, regenerated source by source
    lp_b, _ = g.solve_sources(kappa, mu, lp_solver, rho_lp, seed, 0, n_lp, nrhs_per_launch=nb)
    lp_c, _ = g.solve_sources(kappa, mu, lp_solver, rho_lp, seed, n_lp, n_hp, nrhs_per_launch=nb)
    # contracted in the driver's batches (FP32 source sums per batch, FP64 across batches)
    fs = g.native_bytes(abi.TSM_F32, 1)
    acc = None
    for k0 in range(0, n_lp, nb):
        acc = g.contract(kappa, mu, abi.TSM_F32, lp_b[k0 * fs:(k0 + nb) * fs], nb, moms, out=acc, accumulate=k0 > 0)
    mine_b = api.loops_complex(acc)
    mine_c = api.loops_complex(g.contract(kappa, mu, abi.TSM_F32, lp_c, n_hp, moms))
    assert _rel(mine_b, parts[0]) < 1e-12 and _rel(mine_c, parts[2]) < 1e-12
    xb = g.unpack(lp_b, abi.TSM_F32, n_lp).cpu().numpy()
    xc = g.unpack(lp_c, abi.TSM_F32, n_hp).cpu().numpy()
    eo = bool(lp_solver & EO)
    bulk = 0
    for r in range(n_lp):
        eta = philox.z4_source(dims, seed, r)
        assert _normal_residual(u, eta, xb[r], dims, kappa, mu, eo) <= rho_lp
        bulk = bulk + contract.project(contract.loop_densities(u, xb[r], kappa, mu), dims, moms)
    lpc, hp = 0, 0
    for k in range(n_hp):
        r = n_lp + k
        eta = philox.z4_source(dims, seed, r)
        assert _normal_residual(u, eta, xc[k], dims, kappa, mu, eo) <= rho_lp
        lpc = lpc + contract.project(contract.loop_densities(u, xc[k], kappa, mu), dims, moms)
        hp = hp + tsm.source_loops(u, dims, kappa, mu, seed, r, 1e-12, moms)[0]
    want = tsm.combine(bulk, n_lp, hp, lpc, n_hp)
    errs = dict(bulk=_rel(parts[0], bulk), lp_corr=_rel(parts[2], lpc), hp=_rel(parts[1], hp), est=_rel(est, want))
    assert all(v < TOL for v in errs.values()), errs


def test_tsm_consistent_with_exact_traces(ctx):
    """E_TSM - Tr[X (G_u -/+ G_d)] within 4 sigma (variance of the TSM mean
    from the per-source samples), with a crude FP16 LP map (rho = 0.3) whose
    LP-only mean misses the exact value; p = 0, scalar and g5 insertions of
    both flavour structures, every timeslice."""
    dims = (2, 2, 2, 4)
    kappa, mu, seed = 0.12, 0.1, 1303
    lp_solver, hp_solver = abi.TSM_SOLVER_LP_F16 | EO, abi.TSM_SOLVER_F32_RELIABLE | EO
    g, links = gauge(ctx, dims, 0.4, 51, -1)
    u = lattice.effective_links(links, -1)
    moms = [(0, 0, 0)]
    exact = contract.project(dense.exact_flavour_densities(u, dims, kappa, mu), dims, moms)
    n_lp, n_hp, rho_lp = 400, 200, 0.3
    est, st = g.tsm(kappa, mu, n_lp, n_hp, rho_lp, 1e-8, lp_solver, hp_solver, seed, moms, nrhs_per_launch=32)
    assert st["n_not_converged"] == 0

    def per_source(solver_kind, rho, first, n):
        nat, _ = g.solve_sources(kappa, mu, solver_kind, rho, seed, first, n, nrhs_per_launch=32)
        prec = api.solution_prec(solver_kind)
        if prec != abi.TSM_F32:  # the driver contracts every map's solutions in FP32
            nat = g.pack(g.unpack(nat, prec, n), abi.TSM_F32)
        fs = g.native_bytes(abi.TSM_F32, 1)
        return np.array([api.loops_complex(g.contract(kappa, mu, abi.TSM_F32, nat[k * fs:(k + 1) * fs], 1, moms))
                         for k in range(n)])

    lp = per_source(lp_solver, rho_lp, 0, n_lp + n_hp)
    hp = per_source(hp_solver, 1e-8, n_lp, n_hp)
    corr = hp - lp[n_lp:]
    # the driver contracts batches of 32 (FP32 source sums within a batch): same estimate to FP32 rounding
    assert np.abs(tsm.combine(lp[:n_lp].sum(0), n_lp, hp.sum(0), lp[n_lp:].sum(0), n_hp) - est).max() \
        <= 1e-5 * np.abs(est).max()

    def var(a):
        return a.real.var(0, ddof=1) + 1j * a.imag.var(0, ddof=1)

    v = var(lp[:n_lp]) / n_lp + var(corr) / n_hp
    sig = np.sqrt(v.real) + 1j * np.sqrt(v.imag)
    lp_only = lp[:n_lp].mean(0)
    v_lp = var(lp[:n_lp]) / n_lp
    biased = 0
    for ins in (0, 15, 80, 95):
        for t in range(dims[3]):
            d = est[ins, 0, t] - exact[ins, 0, t]
            assert abs(d.real) <= 4 * sig[ins, 0, t].real + 1e-12, (ins, t, d, sig[ins, 0, t])
            assert abs(d.imag) <= 4 * sig[ins, 0, t].imag + 1e-12, (ins, t, d, sig[ins, 0, t])
            e = lp_only[ins, 0, t] - exact[ins, 0, t]
            biased += abs(e.real) > 4 * np.sqrt(v_lp[ins, 0, t].real) or abs(e.imag) > 4 * np.sqrt(v_lp[ins, 0, t].imag)
    assert biased > 0  # the crude LP map alone is inconsistent: the correction does the work
