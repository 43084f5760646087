"""Even-odd preconditioned solves (TSM_SOLVER_EO) on the GPU against the oracle.

* F64 | EO runs the same textbook CG on Mhat^dag Mhat as ``oracle.evenodd``
  (x0 = 0, same stopping rule), so iterates agree to rounding: solutions on
  all sites within 1e-9 relative, iteration counts within +-1, and the
  reported residual is the oracle's odd-site normal residual of the returned
  solution.
* The truncated solvers with EO: the defining property -- the odd-site
  normal residual of the returned x, recomputed in FP64 by the oracle, is at
  most rho (the solvers stop a certification margin below rho) -- and
  the error against the oracle's converged solution within cond-style bounds.
* tsm_invert (M and M^dag) and the TSM driver accept the flag; the TSM
  estimate with FP64 | EO maps equals the oracle's TSM to 1e-9.
* Argument checks: odd L[0] and the multi-instance batch refuse the flag.
"""
import numpy as np
import pytest
import torch

from conftest import rel_err
from gpu_helpers import gauge, to_device
from oracle import dirac, evenodd, lattice, momenta, philox, solver, tsm
from paper_1401_6750_gb300 import abi, api, synth

pytestmark = pytest.mark.gpu
EO = abi.TSM_SOLVER_EO


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_eo_f64_follows_oracle_schur_cg(ctx, dims):
    kappa, mu, rho, seed = 0.125, 0.01, 1e-10, 1101
    g, links = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    u = lattice.effective_links(links, -1)
    n = 4
    nat, stats = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64 | EO, rho, seed, 0, n, nrhs_per_launch=3)
    x = g.unpack(nat, abi.TSM_F64, n).cpu().numpy()
    for k in range(n):
        eta = philox.z4_source(dims, seed, k)
        want, iters, res = evenodd.solve(u, eta, dims, kappa, mu, rho)
        assert stats[k]["converged"] == 1
        assert abs(stats[k]["iterations"] - iters) <= 1, (stats[k], iters)
        assert rel_err(x[k], want) < 1e-9
        assert stats[k]["true_residual"] <= rho
        assert abs(evenodd.normal_residual(u, eta, x[k], dims, kappa, mu) - stats[k]["true_residual"]) < 1e-3 * rho
        full = dirac.apply_M(u, x[k], kappa, mu) - eta
        assert np.linalg.norm(full.ravel()) / np.linalg.norm(eta.ravel()) < 1e-8
    g.close()


@pytest.mark.parametrize("solver_kind,rho", [
    (abi.TSM_SOLVER_F32_RELIABLE, 1e-8),
    (abi.TSM_SOLVER_LP_F16, 1e-2),
    (abi.TSM_SOLVER_LP_BF16, 1e-2),
])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 6, 4, 10)])
def test_eo_truncated_solvers_meet_rho(ctx, solver_kind, rho, dims):
    kappa, mu, seed = 0.125, 0.01, 1102
    g, links = gauge(ctx, dims, 0.3, 2, -1)
    u = lattice.effective_links(links, -1)
    n = 5
    nat, stats = g.solve_sources(kappa, mu, solver_kind | EO, rho, seed, 3, n, nrhs_per_launch=2)
    x = g.unpack(nat, api.solution_prec(solver_kind), n).cpu().numpy()
    for k in range(n):
        eta = philox.z4_source(dims, seed, 3 + k)
        assert stats[k]["converged"] == 1, stats[k]
        assert stats[k]["true_residual"] <= rho
        res = evenodd.normal_residual(u, eta, x[k], dims, kappa, mu)
        assert res <= rho, (res, stats[k])
        exact, _, _ = solver.solve(u, eta, kappa, mu, 1e-12)
        assert rel_err(x[k], exact) < 1e4 * rho
    g.close()


def test_eo_needs_fewer_iterations(ctx):
    dims = (8, 6, 4, 10)
    kappa, mu, seed = 0.125, 0.01, 1103
    g, _ = gauge(ctx, dims, 0.3, 3, -1, precs=(abi.TSM_F64,))
    _, plain = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64, 1e-8, seed, 0, 2)
    _, eo = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64 | EO, 1e-8, seed, 0, 2)
    for a, b in zip(plain, eo):
        assert b["iterations"] < a["iterations"], (a, b)
    g.close()


def test_eo_invert_caller_rhs_and_adjoint(ctx):
    dims = (4, 4, 2, 6)
    kappa, mu = 0.12, 0.05
    g, links = gauge(ctx, dims, 0.4, 9, -1)
    u = lattice.effective_links(links, -1)
    b = synth.gaussian_spinor(dims, 10, nrhs=2)
    for solver_kind in (abi.TSM_SOLVER_F64, abi.TSM_SOLVER_F32_RELIABLE):
        nb = g.pack(to_device(b), abi.TSM_F64)
        bq = g.unpack(nb, abi.TSM_F64, 2).cpu().numpy()
        for op in (abi.TSM_OP_M, abi.TSM_OP_MDAG):
            nx, st = g.invert(op, kappa, mu, solver_kind | EO, 1e-11, nb, 2)
            x = g.unpack(nx, abi.TSM_F64, 2).cpu().numpy()
            apply = dirac.apply_M if op == abi.TSM_OP_M else dirac.apply_Mdag
            for r in range(2):
                assert rel_err(apply(u, x[r], kappa, mu), bq[r]) < 1e-9, (solver_kind, op)
    g.close()


def test_eo_tsm_f64_maps_match_oracle(ctx):
    dims = (4, 4, 4, 4)
    kappa, mu, seed = 0.125, 0.01, 1104
    g, links = gauge(ctx, dims, 0.3, 1, -1)
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    n_lp, n_hp = 4, 2
    est, parts, st = g.tsm(kappa, mu, n_lp, n_hp, 1e-11, 1e-11, abi.TSM_SOLVER_F64 | EO, abi.TSM_SOLVER_F64 | EO,
                           seed, moms, nrhs_per_launch=3, want_parts=True)
    # both maps converged far below the statistical level: the oracle's
    # tightly converged solves of the same sources give the same sums
    want, (bulk, hp, lpc) = tsm.tsm_loops(u, dims, kappa, mu, seed, n_lp, n_hp, 1e-12, 1e-12, moms)
    for got, ref in ((parts[0], bulk), (parts[1], hp), (parts[2], lpc), (est[None], want[None])):
        got, ref = np.asarray(got), np.asarray(ref)
        assert np.linalg.norm((got - ref).ravel()) <= 1e-8 * np.linalg.norm(ref.ravel())
    assert st["n_not_converged"] == 0
    g.close()


def test_eo_tsm_lowprec(ctx):
    dims = (6, 4, 4, 8)
    kappa, mu, seed = 0.125, 0.01, 1105
    g, links = gauge(ctx, dims, 0.3, 2, -1)
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    n_lp, n_hp = 8, 3
    est, parts, st = g.tsm(kappa, mu, n_lp, n_hp, 1e-2, 1e-10, abi.TSM_SOLVER_LP_F16 | EO,
                           abi.TSM_SOLVER_F32_RELIABLE | EO, seed, moms, nrhs_per_launch=4, want_parts=True)
    assert np.allclose(est, parts[0] / n_lp + (parts[1] - parts[2]) / n_hp, rtol=1e-12, atol=1e-14)
    hp = 0
    for r in range(n_lp, n_lp + n_hp):
        hp = hp + tsm.source_loops(u, dims, kappa, mu, seed, r, 1e-12, moms)[0]
    rel = max(np.linalg.norm(parts[1][i] - hp[i]) / np.linalg.norm(hp[i]) for i in range(hp.shape[0]))
    assert rel < 1e-6  # FP32 HP solves: 1e-6
    assert st["n_not_converged"] == 0
    g.close()


def test_eo_argument_checks(ctx):
    for dims in ((3, 4, 2, 4), (4, 4, 2, 5), (4, 3, 2, 4)):
        g, _ = gauge(ctx, dims, 0.3, 1, -1)
        with pytest.raises(abi.TsmError) as e:
            g.solve_sources(0.125, 0.01, abi.TSM_SOLVER_F64 | EO, 1e-8, 1, 0, 1)
        assert e.value.code == abi.TSM_ERR_INVALID_ARG
        g.close()
    g, _ = gauge(ctx, (4, 4, 2, 4), 0.3, 1, -1)
    inst = dict(gauge=g, kappa=0.125, mu=0.01, noise_seed=1, first_src=0, nsrc=1)
    with pytest.raises(abi.TsmError):
        api.solve_batch([inst], abi.TSM_SOLVER_F64 | EO, 1e-8)
    g.close()


@pytest.mark.parametrize("solver_kind", [abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_LP_BF16, abi.TSM_SOLVER_F32_RELIABLE])
def test_eo_map_independent_of_batch(ctx, solver_kind):
    """Each source's solution is the same bits whatever batch it is solved in
    (alone, in a partial group of the shared-link hop, in groups of 8): the
    truncated solver method needs one LP map for bulk and correction sources."""
    dims = (6, 4, 4, 8)
    g, _ = gauge(ctx, dims, 0.3, 4, -1)
    prec = api.solution_prec(solver_kind)
    rho = 1e-2 if solver_kind != abi.TSM_SOLVER_F32_RELIABLE else 1e-8
    fs = g.native_bytes(prec, 1)
    ref = [g.solve_sources(0.125, 0.01, solver_kind | EO, rho, 1106, k, 1)[0] for k in range(13)]
    for nb in (3, 8, 13):
        sol, _ = g.solve_sources(0.125, 0.01, solver_kind | EO, rho, 1106, 0, 13, nrhs_per_launch=nb)
        for k in range(13):
            assert torch.equal(sol[k * fs:(k + 1) * fs], ref[k]), (nb, k)
    g.close()


@pytest.mark.parametrize("solver_kind", [abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_F32_RELIABLE, abi.TSM_SOLVER_F64])
def test_eo_generated_sources_match_explicit(ctx, solver_kind):
    """tsm_solve_sources generates its Z4 sources split by parity, with
    M_ee^-1 eta_e, in one kernel; tsm_invert on the same sources made by
    tsm_make_sources splits and scales them in another.  Every component
    involved is exact (Z4 entries, +-cr and +-ci), so both give the same
    solution values."""
    dims = (6, 4, 4, 8)
    g, _ = gauge(ctx, dims, 0.3, 4, -1)
    prec = api.solution_prec(solver_kind)
    rho = 1e-2 if solver_kind == abi.TSM_SOLVER_LP_F16 else 1e-8
    eta = g.sources(1107, 3, 4, prec)
    a, _ = g.invert(abi.TSM_OP_M, 0.125, 0.01, solver_kind | EO, rho, eta, 4)
    b, _ = g.solve_sources(0.125, 0.01, solver_kind | EO, rho, 1107, 3, 4)
    assert torch.equal(g.unpack(a, prec, 4), g.unpack(b, prec, 4))
    g.close()
