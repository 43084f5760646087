"""Degenerate cases of the path on the GPU.

* Zero twisted mass: the tau_3 loops (insertions 0..79, prefactor -2 i mu')
  vanish exactly, and the loops without tau_3 still match the oracle's
  literal densities (FP64 1e-11, FP32 1e-6).
* A zero right-hand side: every solver returns x = 0 exactly, reports it
  converged after 0 iterations with a zero residual, and its batch mates are
  unaffected (they match the same solve run alone, bit for bit).
* Empty batches: zero sources contract to zero loops (or leave an
  accumulator untouched) and solve to nothing, without touching the device
  buffers; negative counts are refused.
"""
import numpy as np
import pytest

from gpu_helpers import gauge, round_to, to_device
from oracle import contract, lattice, momenta
from paper_1401_6750_gb300 import abi, api, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(abi.TSM_F64, 1e-11), (abi.TSM_F32, 1e-6)])
def test_tau3_loops_vanish_at_zero_twisted_mass(ctx, prec, tol):
    dims, kappa, mu = (4, 4, 4, 6), 0.125, 0.0
    g, links = gauge(ctx, dims, 0.3, 6, -1)
    u = lattice.effective_links(links, -1)
    s = round_to(synth.gaussian_spinor(dims, 61, nrhs=2), prec)
    moms = momenta.momentum_list(4)
    out = api.loops_complex(g.contract(kappa, mu, prec, g.pack(to_device(s), prec), 2, moms))
    assert np.all(out[:80] == 0)
    want = sum(contract.project(contract.loop_densities(u, s[r], kappa, mu), dims, moms) for r in range(2))
    assert np.all(want[:80] == 0)  # the oracle's own prefactor
    for ins in range(80, 160):
        err = np.linalg.norm(out[ins] - want[ins]) / np.linalg.norm(want[ins])
        assert err < tol, (ins, err)
    g.close()


@pytest.mark.parametrize("solver_kind,eo", [(abi.TSM_SOLVER_F64, 0), (abi.TSM_SOLVER_F32_RELIABLE, 0),
                                            (abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_EO),
                                            (abi.TSM_SOLVER_F32_RELIABLE, abi.TSM_SOLVER_EO)])
def test_zero_right_hand_side(ctx, solver_kind, eo):
    dims, kappa, mu = (4, 4, 4, 4), 0.125, 0.01
    g, _ = gauge(ctx, dims, 0.3, 7, -1)
    prec = api.solution_prec(solver_kind)
    b = synth.gaussian_spinor(dims, 62, nrhs=3)
    b[1] = 0.0
    rho = 1e-2 if solver_kind == abi.TSM_SOLVER_LP_F16 else 1e-8
    nb = g.pack(to_device(b), prec)  # b in the solver's output precision
    nx, st = g.invert(abi.TSM_OP_M, kappa, mu, solver_kind | eo, rho, nb, 3)
    x = g.unpack(nx, prec, 3).cpu().numpy()
    assert np.all(x[1] == 0)
    assert st[1]["converged"] == 1 and st[1]["iterations"] == 0 and st[1]["true_residual"] == 0
    for r in (0, 2):
        assert st[r]["converged"] == 1 and st[r]["true_residual"] <= rho
        alone, _ = g.invert(abi.TSM_OP_M, kappa, mu, solver_kind | eo, rho, g.pack(to_device(b[r:r + 1]), prec), 1)
        assert np.array_equal(g.unpack(alone, prec, 1).cpu().numpy()[0], x[r])
    g.close()


def test_empty_batches(ctx):
    import ctypes
    import torch
    dims = (4, 4, 4, 4)
    g, _ = gauge(ctx, dims, 0.3, 8, -1)
    moms = np.ascontiguousarray(np.array(momenta.momentum_list(1), dtype=np.int32))
    nat = g.empty_native(abi.TSM_F64, 1)
    out = torch.full((abi.TSM_N_INSERTIONS, moms.shape[0], dims[3], 2), 7.0, dtype=torch.float64, device="cuda")
    lib = abi.lib()
    mom_p = moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def contract(nsrc, accumulate):
        return lib.tsm_contract_loops(g.handle, 0.125, 0.01, abi.TSM_F64, ctypes.c_void_p(nat.data_ptr()), nsrc,
                                      moms.shape[0], mom_p, ctypes.c_void_p(out.data_ptr()), accumulate, stream)
    assert contract(0, 1) == abi.TSM_OK  # accumulate nothing: untouched
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    assert contract(0, 0) == abi.TSM_OK  # zero sources: zero loops
    torch.cuda.synchronize()
    assert torch.all(out == 0.0)
    assert contract(-1, 0) == abi.TSM_ERR_INVALID_ARG
    sentinel = torch.full((16,), 3.0, dtype=torch.float64, device="cuda")
    rc = lib.tsm_solve_sources(g.handle, 0.125, 0.01, abi.TSM_SOLVER_F64, 1e-8, 100, 1, 0, 0, 0,
                               ctypes.c_void_p(sentinel.data_ptr()), None, stream)
    assert rc == abi.TSM_OK
    torch.cuda.synchronize()
    assert torch.all(sentinel == 3.0)
    g.close()


@pytest.mark.parametrize("prec,tol", [(abi.TSM_F64, 1e-11), (abi.TSM_F32, 1e-6)])
def test_largest_momentum_radius(ctx, prec, tol):
    """Momentum components up to the accepted maximum |n| = 8 (the x/y
    transform then keeps 17 x 17 partial sums per field), larger than the
    extents (the phases alias), against the oracle's direct Fourier sums;
    |n| = 9 is refused."""
    dims, kappa, mu = (6, 4, 8, 4), 0.125, 0.01
    g, links = gauge(ctx, dims, 0.3, 9, -1)
    u = lattice.effective_links(links, -1)
    s = round_to(synth.gaussian_spinor(dims, 63, nrhs=2), prec)
    moms = [(8, 0, 0), (-8, 3, 0), (0, 8, -8), (5, -7, 2), (0, 0, 0)]
    nat = g.pack(to_device(s), prec)
    out = api.loops_complex(g.contract(kappa, mu, prec, nat, 2, moms))
    want = sum(contract.project(contract.loop_densities(u, s[r], kappa, mu), dims, moms) for r in range(2))
    for ins in range(160):
        err = np.linalg.norm(out[ins] - want[ins]) / np.linalg.norm(want[ins])
        assert err < tol, (ins, err)
    with pytest.raises(abi.TsmError):
        g.contract(kappa, mu, prec, nat, 2, [(9, 0, 0)])
    g.close()


@pytest.mark.parametrize("solver_kind,eo,bad", [(abi.TSM_SOLVER_F64, 0, np.nan),
                                                (abi.TSM_SOLVER_LP_F16, abi.TSM_SOLVER_EO, np.inf),
                                                (abi.TSM_SOLVER_F32_RELIABLE, abi.TSM_SOLVER_EO, np.nan)])
def test_nonfinite_right_hand_side_reported(ctx, solver_kind, eo, bad):
    """A NaN or Inf in a caller's right-hand side ends that right-hand side's
    CG as a breakdown (its |b|^2 is not finite) and the call returns
    TSM_ERR_NONFINITE, without hanging."""
    dims, kappa, mu = (4, 4, 4, 4), 0.125, 0.01
    g, _ = gauge(ctx, dims, 0.3, 10, -1)
    prec = api.solution_prec(solver_kind)
    b = synth.gaussian_spinor(dims, 64, nrhs=2)
    b[1].flat[17] = bad
    nb = g.pack(to_device(b), prec)
    with pytest.raises(abi.TsmError) as e:
        g.invert(abi.TSM_OP_M, kappa, mu, solver_kind | eo, 1e-2, nb, 2)
    assert e.value.code == abi.TSM_ERR_NONFINITE
    g.close()
