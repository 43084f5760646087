"""The tensor-core checkerboarded hop (16-bit fields, batches of >= 8
right-hand sides; opt-in with TSM_TC_HOP=1) against the FP64 oracle.

The library reads the switch once per process, so the tensor-core cases run
in child processes; the same checks run in this process on the default
(CUDA-core) path, at the same batch shape.

* Schur operator Mhat and Mhat^dag, FP16 and BF16, 10 right-hand sides (a
  full group of 8 and a ragged group of 2), on lattices with several tiles
  and a ragged tail of sites, both boundary conditions: element-wise against
  ``oracle.evenodd`` with the tolerance of the CUDA-core path
  (test_gpu_dslash: two half-volume hops with a stored 16-bit intermediate).
  The tensor-core path also rounds the rebuilt third link row to the 16-bit
  type, an error of the same order as the stored rows'.
* Even-odd LP solves, FP16 and BF16, 10 sources in one batch: every returned
  solution meets its defining property, the odd-site normal residual
  recomputed in FP64 by the oracle at most rho.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL_MHAT = {2: 6e-3, 3: 6e-2}  # TSM_F16, TSM_BF16
RHO = 1e-2

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
from gpu_helpers import gauge, round_to, to_device
from oracle import evenodd, lattice, philox
from paper_1401_6750_gb300 import abi, api, synth
ctx = api.Context(0)
out = {"operator": [], "solve": []}
kappa, mu, nrhs = 0.13, 0.07, 10
for dims in ((8, 6, 4, 10), (6, 4, 2, 8), (4, 4, 4, 4)):
    for t_bc in (-1, 1):
        g, links = gauge(ctx, dims, 0.35, 23, t_bc)
        u = lattice.effective_links(links, t_bc)
        for prec in (abi.TSM_F16, abi.TSM_BF16):
            psi = round_to(synth.gaussian_spinor(dims, 24, nrhs=nrhs), prec)
            nat = g.pack(to_device(psi), prec)
            for op, fn in ((abi.TSM_OP_MHAT, evenodd.apply_mhat), (abi.TSM_OP_MHATDAG, evenodd.apply_mhat_dag)):
                got = g.unpack(g.dslash(op, kappa, mu, prec, nat, nrhs), prec, nrhs).cpu().numpy()
                for r in range(nrhs):
                    want = fn(u, psi[r], dims, kappa, mu)
                    out["operator"].append([list(dims), t_bc, prec, op, r,
                        float(np.linalg.norm((got[r] - want).ravel()) / np.linalg.norm(want.ravel())),
                        float(np.max(np.abs(got[r] - want)) / np.max(np.abs(want))),
                        bool(np.all(evenodd.restrict(got[r], dims, 0) == 0))])
        g.close()
dims, kappa, mu, seed, n = (8, 6, 4, 10), 0.125, 0.01, 1202, 10
g, links = gauge(ctx, dims, 0.3, 4, -1)
u = lattice.effective_links(links, -1)
for kind in (abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_LP_BF16):
    nat, stats = g.solve_sources(kappa, mu, kind | abi.TSM_SOLVER_EO, RHO, seed, 0, n, nrhs_per_launch=n)
    x = g.unpack(nat, api.solution_prec(kind), n).cpu().numpy()
    for k in range(n):
        res = evenodd.normal_residual(u, philox.z4_source(dims, seed, k), x[k], dims, kappa, mu)
        out["solve"].append([kind, k, float(res), int(stats[k]["converged"]), float(stats[k]["true_residual"])])
g.close()
ctx.close()
print("RESULT " + json.dumps(out))
"""


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    code = "ROOT = %r\nRHO = %r\n" % (ROOT, RHO) + CHILD
    proc = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=1200)
    assert proc.returncode == 0, proc.stdout[-2000:] + proc.stderr[-4000:]
    return json.loads([ln for ln in proc.stdout.splitlines() if ln.startswith("RESULT ")][-1][len("RESULT "):])


@pytest.mark.parametrize("tc", ["1", "0"])
def test_schur_operator_and_lp_solves_large_batch(ctx, tc):
    res = _run({"TSM_TC_HOP": tc})
    assert len(res["operator"]) == 3 * 2 * 2 * 2 * 10
    for dims, t_bc, prec, op, r, norm_err, max_err, even_zero in res["operator"]:
        tol = TOL_MHAT[prec]
        assert norm_err < tol, (tc, dims, t_bc, prec, op, r, norm_err)
        assert max_err <= 4 * tol, (tc, dims, t_bc, prec, op, r, max_err)
        assert even_zero
    assert len(res["solve"]) == 2 * 10
    for kind, k, r, conv, true_res in res["solve"]:
        assert conv == 1
        assert true_res <= RHO
        assert r <= RHO, (tc, kind, k, r)
