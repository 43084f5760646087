"""Binary-weight accumulation on the GPU (Sec. 2.1.1, Fig. 2): the block
driver computes the bulk LP loops block by block, and any N read back equals
the mean over the oracle-selected sources of the library's own per-source
loops (FP64 maps: 1e-12; sums over a batch differ only in rounding order) and
the oracle's loops (1e-9).  An interrupted accumulation resumes from the
blocks on disk and gives the same blocks."""
import numpy as np
import pytest

from gpu_helpers import gauge
from oracle import binstore as obs
from oracle import contract, lattice, momenta, philox, solver
from paper_1401_6750_gb300 import abi, api

pytestmark = pytest.mark.gpu


def test_accumulate_blocks_resume_and_any_n(ctx, tmp_path):
    dims = (4, 4, 4, 4)
    kappa, mu, seed = 0.125, 0.01, 1501
    g, links = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    u = lattice.effective_links(links, -1)
    moms = momenta.momentum_list(9)
    T = dims[3]
    shape = (160, len(moms), T)
    n_values = 160 * len(moms) * T * 2
    st = api.BinStore(tmp_path / "bulk", n_values)
    st.accumulate(g, kappa, mu, abi.TSM_SOLVER_F64, 1e-10, seed, moms, k_end=2, nrhs_per_launch=4)
    assert st.sources == 3
    st.close()
    st = api.BinStore(tmp_path / "bulk", n_values)  # resume after the "interruption"
    stats = st.accumulate(g, kappa, mu, abi.TSM_SOLVER_F64, 1e-10, seed, moms, k_end=3, nrhs_per_launch=4)
    assert st.sources == 7 and stats["n_not_converged"] == 0
    nat, _ = g.solve_sources(kappa, mu, abi.TSM_SOLVER_F64, 1e-10, seed, 0, 7, nrhs_per_launch=4)
    field = g.native_bytes(abi.TSM_F64, 1)
    per = [api.loops_complex(g.contract(kappa, mu, abi.TSM_F64, nat[j * field:(j + 1) * field], 1, moms))
           for j in range(7)]
    for n in range(1, 8):
        a = st.mean(n).reshape(shape + (2,))
        got = a[..., 0] + 1j * a[..., 1]
        want = sum(per[i] for i in obs.sources_for(n)) / n
        assert np.linalg.norm((got - want).ravel()) <= 1e-12 * np.linalg.norm(want.ravel()), n
    want = 0
    for r in range(7):
        s, _, _ = solver.solve(u, philox.z4_source(dims, seed, r), kappa, mu, 1e-10)
        want = want + contract.project(contract.loop_densities(u, s, kappa, mu), dims, moms)
    a = st.mean(7).reshape(shape + (2,))
    got = a[..., 0] + 1j * a[..., 1]
    assert np.linalg.norm((got - want / 7).ravel()) <= 1e-9 * np.linalg.norm((want / 7).ravel())
    st.close()
    g.close()
