"""Uneven batch (several lattices and twisted masses, one launch per CG
kernel) against solving each instance alone.

The per-right-hand-side arithmetic of the batched solver is that of the
single-instance solver (same stencil, same fixed-order reductions over the
instance's own blocks), so the solutions agree to rounding (1e-12 relative;
in practice bit for bit) and the iteration counts are equal.  The instances
are lattices 8^4, 16^3 x 32 and 24^3 x 48 with mu in {0.003, 0.006, 0.01}
(eps 0.3, gauge seeds 4, 5, 6), low-precision rho = 1e-2 solves.
"""
import numpy as np
import pytest

from gpu_helpers import gauge
from paper_1401_6750_gb300 import abi, api

pytestmark = pytest.mark.gpu

LATTICES = [((8, 8, 8, 8), 4), ((16, 16, 16, 32), 5), ((24, 24, 24, 48), 6)]
MUS = (0.003, 0.006, 0.01)


@pytest.mark.parametrize("solver", [abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_F32_RELIABLE])
def test_batch_equals_single_instance_solves(ctx, solver):
    nsrc = 4 if solver == abi.TSM_SOLVER_LP_F16 else 2
    rho = 1e-2 if solver == abi.TSM_SOLVER_LP_F16 else 1e-8
    gauges = [gauge(ctx, dims, 0.3, seed, -1)[0] for dims, seed in LATTICES]
    inst = []
    for g in gauges:
        for j, mu in enumerate(MUS):
            inst.append({"gauge": g, "kappa": 0.125, "mu": mu, "noise_seed": 1004, "first_src": 16 * j,
                         "nsrc": nsrc})
    res = api.solve_batch(inst, solver, rho)
    prec = api.solution_prec(solver)
    for it, (out, st) in zip(inst, res):
        g = it["gauge"]
        ref, st_ref = g.solve_sources(it["kappa"], it["mu"], solver, rho, it["noise_seed"], it["first_src"], nsrc,
                                      nrhs_per_launch=nsrc)
        a = g.unpack(out, prec, nsrc).cpu().numpy()
        b = g.unpack(ref, prec, nsrc).cpu().numpy()
        assert np.linalg.norm((a - b).ravel()) <= 1e-12 * np.linalg.norm(b.ravel())
        for x, y in zip(st, st_ref):
            assert x["converged"] == 1 and x["true_residual"] <= rho
            assert x["iterations"] == y["iterations"]
    for g in gauges:
        g.close()


def test_uneven_batch_64_sources_each(ctx):
    """The full uneven configuration: 9 instances x 64 Z4 sources, LP FP16."""
    gauges = [gauge(ctx, dims, 0.3, seed, -1, precs=(abi.TSM_F32, abi.TSM_F16))[0] for dims, seed in LATTICES]
    inst = [{"gauge": g, "kappa": 0.125, "mu": mu, "noise_seed": 1004, "first_src": 0, "nsrc": 64}
            for g in gauges for mu in MUS]
    res = api.solve_batch(inst, abi.TSM_SOLVER_LP_F16, 1e-2)
    for out, st in res:
        assert all(x["converged"] == 1 and x["true_residual"] <= 1e-2 for x in st)
    for g in gauges:
        g.close()
