"""Stencils that carry several right-hand sides per thread, against the oracle.

The autotuner and the solvers choose one right-hand side per thread at the
shapes the other tests use, so the two- and four-wide forms of the packed-pair
stencils (each link loaded once for all of a thread's right-hand sides, with
inactive slots for a ragged last group) would go untested.  The environment
switches TSM_DSLASH_NR and TSM_EO_NR_F16 / TSM_EO_NR_F32 force them; the
library reads them once per process, so each case runs in a child process.

* Operator M and M^dag, FP32 and FP16 fields, 5 right-hand sides (groups of
  2 + 2 + 1 or 4 + 1): element-wise against the FP64 oracle with the
  storage-type tolerances of test_gpu_dslash.
* Even-odd truncated solves with the sloppy operator at 2 or 4 right-hand
  sides per thread: the odd-site normal residual of every returned solution,
  recomputed in FP64 by the oracle, is at most rho.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

OPERATOR_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
from gpu_helpers import gauge, round_to, to_device
from oracle import dirac, lattice
from paper_1401_6750_gb300 import abi, api, synth
ctx = api.Context(0)
dims, kappa, mu, nrhs = (6, 4, 2, 8), 0.13, 0.04, 5
out = {}
for prec in (abi.TSM_F32, abi.TSM_F16):
    g, links = gauge(ctx, dims, 0.5, 17, -1)
    u = lattice.effective_links(links, -1)
    psi = round_to(synth.gaussian_spinor(dims, 18, nrhs=nrhs), prec)
    nat = g.pack(to_device(psi), prec)
    for op, ref in ((abi.TSM_OP_M, dirac.apply_M), (abi.TSM_OP_MDAG, dirac.apply_Mdag)):
        got = g.unpack(g.dslash(op, kappa, mu, prec, nat, nrhs), prec, nrhs).cpu().numpy()
        errs = []
        for r in range(nrhs):
            want = ref(u, psi[r], kappa, mu)
            errs.append([float(np.linalg.norm((got[r] - want).ravel()) / np.linalg.norm(want.ravel())),
                         float(np.max(np.abs(got[r] - want)) / np.max(np.abs(want)))])
        out["%d_%d" % (prec, op)] = errs
    g.close()
ctx.close()
print("RESULT " + json.dumps(out))
"""

SOLVE_CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
from gpu_helpers import gauge
from oracle import evenodd, lattice, philox
from paper_1401_6750_gb300 import abi, api
ctx = api.Context(0)
dims, kappa, mu, seed, n = (8, 6, 4, 10), 0.125, 0.01, 1102, 5
g, links = gauge(ctx, dims, 0.3, 2, -1)
u = lattice.effective_links(links, -1)
out = {}
for kind, rho in ((abi.TSM_SOLVER_LP_F16, 1e-2), (abi.TSM_SOLVER_F32_RELIABLE, 1e-8)):
    nat, stats = g.solve_sources(kappa, mu, kind | abi.TSM_SOLVER_EO, rho, seed, 3, n, nrhs_per_launch=n)
    x = g.unpack(nat, api.solution_prec(kind), n).cpu().numpy()
    res = []
    for k in range(n):
        eta = philox.z4_source(dims, seed, 3 + k)
        res.append([float(evenodd.normal_residual(u, eta, x[k], dims, kappa, mu)), int(stats[k]["converged"])])
    out[str(kind)] = res
g.close()
ctx.close()
print("RESULT " + json.dumps(out))
"""


def _run(code, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    proc = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + code], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=900)
    assert proc.returncode == 0, proc.stdout[-2000:] + proc.stderr[-4000:]
    line = [ln for ln in proc.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


@pytest.mark.parametrize("nr", ["2", "4"])
def test_operator_rhs_per_thread(ctx, nr):
    from paper_1401_6750_gb300 import abi
    tol = {abi.TSM_F32: 2e-6, abi.TSM_F16: 3e-3}
    res = _run(OPERATOR_CHILD, {"TSM_DSLASH_NR": nr})
    for key, errs in res.items():
        prec = int(key.split("_")[0])
        for norm_err, max_err in errs:
            assert norm_err < tol[prec], (nr, key, norm_err)
            assert max_err <= 4 * tol[prec], (nr, key, max_err)


@pytest.mark.parametrize("env", [{"TSM_EO_NR_F16": "4", "TSM_EO_NR_F32": "2"},
                                 {"TSM_EO_NR_F16": "2", "TSM_EO_NR_F32": "4"}])
def test_eo_solves_rhs_per_thread(ctx, env):
    from paper_1401_6750_gb300 import abi
    res = _run(SOLVE_CHILD, env)
    for kind, rho in ((abi.TSM_SOLVER_LP_F16, 1e-2), (abi.TSM_SOLVER_F32_RELIABLE, 1e-8)):
        for r, conv in res[str(kind)]:
            assert conv == 1
            assert r <= rho, (env, kind, r)
