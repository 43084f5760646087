"""Truncated Solver Method end to end (Sec. 2.1) against the oracle.

* With FP64 low- and high-precision maps the GPU TSM and the oracle TSM run
  the same CG on the same Z4 sources, so the combined 160 x 123 x T estimate
  agrees to 1e-9 (normwise per insertion).
* With the 16-bit LP map the estimate depends on the (non-unique) LP
  solutions; what is unique -- the combine identity over the returned
  per-set sums, and the HP-set sum, which only depends on solves to
  rho_HP -- is checked.
* The plain method of the first configuration: 4^4, eps 0.3, seed 1,
  kappa 0.125, mu 0.01, 4 Z4 sources, FP64 CG to 1e-8, 16 ultra-local loops at
  p = 0 per timeslice, within 1e-9 of the oracle.
"""
import numpy as np
import pytest

from gpu_helpers import gauge
from oracle import contract, lattice, momenta, philox, solver, tsm
from paper_1401_6750_gb300 import abi

pytestmark = pytest.mark.gpu


def _norm_rel(got, want):
    return max(np.linalg.norm(got[i] - want[i]) / np.linalg.norm(want[i]) for i in range(want.shape[0]))


def test_tsm_f64_maps_match_oracle(ctx):
    dims = (4, 4, 4, 4)
    kappa, mu, seed = 0.125, 0.01, 1001
    g, links = gauge(ctx, dims, 0.3, 1, -1)
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    n_lp, n_hp, rho_lp, rho_hp = 5, 2, 1e-3, 1e-10
    est, parts, st = g.tsm(kappa, mu, n_lp, n_hp, rho_lp, rho_hp, abi.TSM_SOLVER_F64, abi.TSM_SOLVER_F64, seed,
                           moms, nrhs_per_launch=3, want_parts=True)
    want, (bulk, hp, lpc) = tsm.tsm_loops(u, dims, kappa, mu, seed, n_lp, n_hp, rho_lp, rho_hp, moms)
    assert _norm_rel(parts[0], bulk) < 1e-9
    assert _norm_rel(parts[1], hp) < 1e-9
    assert _norm_rel(parts[2], lpc) < 1e-9
    assert _norm_rel(est, want) < 1e-9
    g.close()


@pytest.mark.parametrize("lp_solver", [abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_LP_BF16])
def test_tsm_lowprec_combine_and_hp_part(ctx, lp_solver):
    dims = (6, 4, 4, 8)
    kappa, mu, seed = 0.125, 0.01, 1002
    g, links = gauge(ctx, dims, 0.3, 2, -1)
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    n_lp, n_hp = 8, 3
    est, parts, st = g.tsm(kappa, mu, n_lp, n_hp, 1e-2, 1e-10, lp_solver, abi.TSM_SOLVER_F32_RELIABLE, seed, moms,
                           nrhs_per_launch=4, want_parts=True)
    # combine identity
    assert np.allclose(est, parts[0] / n_lp + (parts[1] - parts[2]) / n_hp, rtol=1e-12, atol=1e-14)
    # HP part against oracle FP64 solves of the same sources
    hp = 0
    for r in range(n_lp, n_lp + n_hp):
        hp = hp + tsm.source_loops(u, dims, kappa, mu, seed, r, 1e-12, moms)[0]
    assert _norm_rel(parts[1], hp) < 1e-6  # FP32 HP solves: 1e-6
    assert st["lp_max_true_residual"] <= 1e-2 and st["hp_max_true_residual"] <= 1e-10
    assert st["n_not_converged"] == 0
    g.close()


def test_plain_method_4x4x4x4_ultralocal_p0(ctx):
    dims = (4, 4, 4, 4)
    kappa, mu, seed, nsrc = 0.125, 0.01, 1001, 4
    g, links = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    u = lattice.effective_links(links, -1)
    nat, stats = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64, 1e-8, seed, 0, nsrc)
    assert all(s["converged"] and s["true_residual"] <= 1e-8 for s in stats)
    from paper_1401_6750_gb300 import api
    got = api.loops_complex(g.contract(kappa, mu, abi.TSM_F64, nat, nsrc, [(0, 0, 0)])) / nsrc
    want = 0
    for r in range(nsrc):
        s, _, _ = solver.solve(u, philox.z4_source(dims, seed, r), kappa, mu, 1e-8)
        want = want + contract.project(contract.loop_densities(u, s, kappa, mu), dims, [(0, 0, 0)])
    want = want / nsrc
    for ins in list(range(16)) + list(range(80, 96)):
        assert np.linalg.norm(got[ins] - want[ins]) <= 1e-9 * np.linalg.norm(want[ins]), ins
    g.close()
