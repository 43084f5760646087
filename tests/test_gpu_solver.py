"""CG on M^dag M (Eq. 1) on the GPU against the oracle.

* F64: the GPU runs the same textbook CG as the oracle (x0 = 0, same stopping
  rule), so iterates agree to rounding: solutions within 1e-9 relative and
  the same iteration count (+-1).
* F32 with reliable updates and the LP 16-bit solvers: a truncated solve is
  not unique, so what is checked is its defining property -- the true
  residual of the returned x, recomputed by the oracle's FP64 operator, is at
  most rho (the solvers stop a certification margin below rho) -- plus the
  error against the oracle's converged solution within cond-style bounds.
"""
import numpy as np
import pytest

from conftest import rel_err
from gpu_helpers import gauge
from oracle import dirac, lattice, philox, solver
from paper_1401_6750_gb300 import abi, api

pytestmark = pytest.mark.gpu


def _true_residual(u, x, eta, kappa, mu):
    b = dirac.apply_Mdag(u, eta, kappa, mu)
    r = b - dirac.apply_MdagM(u, x, kappa, mu)
    return np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_f64_solver_follows_oracle_cg(ctx, dims):
    kappa, mu, rho, seed = 0.125, 0.01, 1e-8, 1001
    g, links = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    u = lattice.effective_links(links, -1)
    n = 4
    nat, stats = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64, rho, seed, 0, n, nrhs_per_launch=3)
    x = g.unpack(nat, abi.TSM_F64, n).cpu().numpy()
    for k in range(n):
        eta = philox.z4_source(dims, seed, k)
        want, iters, res = solver.solve(u, eta, kappa, mu, rho)
        assert stats[k]["converged"] == 1
        assert abs(stats[k]["iterations"] - iters) <= 1, (stats[k], iters)
        assert rel_err(x[k], want) < 1e-9
        assert stats[k]["true_residual"] <= rho
        assert abs(_true_residual(u, x[k], eta, kappa, mu) - stats[k]["true_residual"]) < 1e-3 * rho
    g.close()


@pytest.mark.parametrize("solver_kind,rho", [
    (abi.TSM_SOLVER_F32_RELIABLE, 1e-8),
    (abi.TSM_SOLVER_LP_F16, 1e-2),
    (abi.TSM_SOLVER_LP_BF16, 1e-2),
])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 6, 4, 10)])
def test_truncated_solvers_meet_rho(ctx, solver_kind, rho, dims):
    kappa, mu, seed = 0.125, 0.01, 1002
    g, links = gauge(ctx, dims, 0.3, 2, -1)
    u = lattice.effective_links(links, -1)
    n = 5
    nat, stats = g.solve_sources(kappa, mu, solver_kind, rho, seed, 3, n, nrhs_per_launch=2)
    x = g.unpack(nat, api.solution_prec(solver_kind), n).cpu().numpy()
    for k in range(n):
        eta = philox.z4_source(dims, seed, 3 + k)
        assert stats[k]["converged"] == 1, stats[k]
        assert stats[k]["true_residual"] <= rho
        res = _true_residual(u, x[k], eta, kappa, mu)
        assert res <= rho, (res, stats[k])
        exact, _, _ = solver.solve(u, eta, kappa, mu, 1e-12)
        assert rel_err(x[k], exact) < 1e4 * rho
    g.close()


def test_invert_caller_rhs_and_adjoint(ctx):
    """tsm_invert with op = M and op = M^dag on caller right-hand sides."""
    from gpu_helpers import to_device
    from paper_1401_6750_gb300 import synth
    dims = (4, 4, 2, 6)
    kappa, mu = 0.12, 0.05
    g, links = gauge(ctx, dims, 0.4, 9, -1)
    u = lattice.effective_links(links, -1)
    b = synth.gaussian_spinor(dims, 10, nrhs=2)
    for solver_kind, prec, tol in ((abi.TSM_SOLVER_F64, abi.TSM_F64, 1e-9),
                                   (abi.TSM_SOLVER_F32_RELIABLE, abi.TSM_F64, 1e-9)):
        nb = g.pack(to_device(b), prec)
        for op in (abi.TSM_OP_M, abi.TSM_OP_MDAG):
            nx, st = g.invert(op, kappa, mu, solver_kind, 1e-10, nb, 2)
            x = g.unpack(nx, prec, 2).cpu().numpy()
            bq = g.unpack(nb, prec, 2).cpu().numpy()
            for r in range(2):
                apply = dirac.apply_M if op == abi.TSM_OP_M else dirac.apply_Mdag
                assert rel_err(apply(u, x[r], kappa, mu), bq[r]) < tol, (solver_kind, op)
    g.close()


def test_max_iter_reports_not_converged(ctx):
    dims = (4, 4, 4, 4)
    g, _ = gauge(ctx, dims, 0.3, 1, -1)
    nat, stats = g.solve_sources(0.125, 0.01, abi.TSM_SOLVER_LP_F16, 1e-6, 5, 0, 2, max_iter=3,
                                 allow_not_converged=True)
    for s in stats:
        assert s["converged"] == 0 and s["iterations"] <= 3 and s["true_residual"] > 1e-6
    g.close()


@pytest.mark.parametrize("eo", [0, abi.TSM_SOLVER_EO])
def test_reliable_update_certifies_below_fp32(ctx, eo):
    """The reliable-update solver's precise operator (float-float, about 44
    significant bits) certifies residuals far below FP32 resolution: at
    rho = 1e-10 the oracle's FP64 residual of the returned solution agrees
    with the reported one to 10% of rho (the float-float rounding, amplified
    by |x| / |b| of this system, is a few 1e-12)."""
    from oracle import evenodd
    dims = (4, 4, 4, 6)
    kappa, mu, seed, rho = 0.125, 0.01, 1201, 1e-10
    g, links = gauge(ctx, dims, 0.3, 12, -1, precs=(abi.TSM_F64, abi.TSM_F32))
    u = lattice.effective_links(links, -1)
    nat, stats = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F32_RELIABLE | eo, rho, seed, 0, 3)
    x = g.unpack(nat, abi.TSM_F64, 3).cpu().numpy()
    for k in range(3):
        eta = philox.z4_source(dims, seed, k)
        assert stats[k]["converged"] == 1 and stats[k]["true_residual"] <= rho
        res = (evenodd.normal_residual(u, eta, x[k], dims, kappa, mu) if eo
               else _true_residual(u, x[k], eta, kappa, mu))
        assert res <= 1.1 * rho, (res, stats[k])
        assert abs(res - stats[k]["true_residual"]) <= 0.1 * rho
    g.close()
