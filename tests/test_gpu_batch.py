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


@pytest.mark.parametrize("solver", [abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_F32_RELIABLE])
def test_batch_residuals_recomputed_by_oracle(ctx, solver):
    """The uneven batch's solutions meet rho by the oracle's own FP64
    operator: every instance of the 8^4 lattice (three twisted masses) and
    the 16^3 x 32 instance at mu = 0.006, each source's true residual
    |M^dag eta - M^dag M x| / |M^dag eta| recomputed from the downloaded x."""
    from oracle import dirac, lattice, philox
    nsrc = 3 if solver == abi.TSM_SOLVER_LP_F16 else 2
    rho = 1e-2 if solver == abi.TSM_SOLVER_LP_F16 else 1e-8
    made = [gauge(ctx, dims, 0.3, seed, -1) for dims, seed in LATTICES[:2]]
    inst = []
    for (g, _), (dims, _) in zip(made, LATTICES[:2]):
        for j, mu in enumerate(MUS):
            inst.append({"gauge": g, "dims": dims, "kappa": 0.125, "mu": mu, "noise_seed": 1005,
                         "first_src": 8 * j, "nsrc": nsrc})
    res = api.solve_batch([{k: v for k, v in it.items() if k != "dims"} for it in inst], solver, rho)
    links = {dims: lk for (_, lk), (dims, _) in zip(made, LATTICES[:2])}
    checked = 0
    for it, (out, st) in zip(inst, res):
        dims = it["dims"]
        if dims == (16, 16, 16, 32) and it["mu"] != 0.006:
            continue
        u = lattice.effective_links(links[dims], -1)
        x = it["gauge"].unpack(out, api.solution_prec(solver), nsrc).cpu().numpy()
        for k in range(nsrc):
            eta = philox.z4_source(dims, 1005, it["first_src"] + k)
            b = dirac.apply_Mdag(u, eta, it["kappa"], it["mu"])
            r = b - dirac.apply_MdagM(u, x[k], it["kappa"], it["mu"])
            res_k = np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel())
            assert st[k]["converged"] == 1 and res_k <= rho, (dims, it["mu"], k, res_k, st[k])
            checked += 1
    assert checked == 4 * nsrc
    for g, _ in made:
        g.close()
