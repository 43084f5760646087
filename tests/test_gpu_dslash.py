"""Eq. 1's operator on the GPU against the FP64 oracle, element by element.

Inputs are the same seeded synthetic fields on both sides; for the 16- and
32-bit paths the oracle receives the spinor already rounded to the storage
type (input preparation), so the comparison isolates the kernel's own error:
link storage (two rows kept, the third rebuilt), FP32 arithmetic and output
rounding.  Tolerances, normwise and per element relative to the largest
element, from the unit roundoff u of the storage type:
    F64 1e-13 (u = 1.1e-16, a few dozen operations)
    F32 2e-6  (u = 6e-8)
    F16 3e-3  (u = 2^-11: output rounding + link rounding, hop terms ~ kappa*8*|psi|)
    BF16 3e-2 (u = 2^-8, same budget)
"""
import numpy as np
import pytest

from gpu_helpers import gauge, round_to, to_device
from oracle import dirac, lattice
from paper_1401_6750_gb300 import abi, synth

pytestmark = pytest.mark.gpu

TOL = {abi.TSM_F64: 1e-13, abi.TSM_F32: 2e-6, abi.TSM_F16: 3e-3, abi.TSM_BF16: 3e-2}
OPS = {
    abi.TSM_OP_M: lambda u, p, k, m: dirac.apply_M(u, p, k, m),
    abi.TSM_OP_MDAG: lambda u, p, k, m: dirac.apply_Mdag(u, p, k, m),
    abi.TSM_OP_A: lambda u, p, k, m: dirac.apply_A(u, p, k),
    abi.TSM_OP_MDAGM: lambda u, p, k, m: dirac.apply_MdagM(u, p, k, m),
}


def _check(got, want, tol):
    err = np.linalg.norm((got - want).ravel()) / np.linalg.norm(want.ravel())
    assert err < tol, err
    assert np.max(np.abs(got - want)) <= 4 * tol * np.max(np.abs(want))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (8, 6, 4, 10), (3, 5, 2, 2)])
@pytest.mark.parametrize("t_bc", [-1, 1])
@pytest.mark.parametrize("prec", [abi.TSM_F64, abi.TSM_F32, abi.TSM_F16, abi.TSM_BF16])
def test_operator_matches_oracle(ctx, dims, t_bc, prec):
    kappa, mu = 0.13, 0.04
    g, links = gauge(ctx, dims, 0.5, 17, t_bc)
    u = lattice.effective_links(links, t_bc)
    nrhs = 3
    psi = round_to(synth.gaussian_spinor(dims, 18, nrhs=nrhs), prec)
    nat = g.pack(to_device(psi), prec)
    for op, ref in OPS.items():
        if op == abi.TSM_OP_MDAGM and prec in (abi.TSM_F16, abi.TSM_BF16):
            tol = 2 * TOL[prec]  # intermediate M psi is stored in the 16-bit type
        else:
            tol = TOL[prec]
        out = g.dslash(op, kappa, mu, prec, nat, nrhs)
        got = g.unpack(out, prec, nrhs).cpu().numpy()
        for r in range(nrhs):
            _check(got[r], ref(u, psi[r], kappa, mu), tol)
    g.close()


def test_operator_full_size_sampled(ctx):
    """24^3 x 48 (the throughput lattice): whole field in FP32 against the oracle."""
    dims = (24, 24, 24, 48)
    kappa, mu = 0.125, 0.005
    g, links = gauge(ctx, dims, 0.25, 3, -1, precs=(abi.TSM_F32, abi.TSM_F16))
    u = lattice.effective_links(links, -1)
    psi = round_to(synth.gaussian_spinor(dims, 5, nrhs=1), abi.TSM_F16)
    for prec in (abi.TSM_F32, abi.TSM_F16):
        nat = g.pack(to_device(psi), prec)
        got = g.unpack(g.dslash(abi.TSM_OP_M, kappa, mu, prec, nat, 1), prec, 1).cpu().numpy()[0]
        _check(got, dirac.apply_M(u, psi[0], kappa, mu), TOL[prec])
    g.close()


def test_rejects_bad_arguments(ctx):
    dims = (4, 4, 4, 4)
    g, _ = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F32,))
    x = g.empty_native(abi.TSM_F32, 1)
    lib = abi.lib()
    # missing link precision
    assert lib.tsm_dslash_tm(g.handle, 0.1, 0.1, 0, abi.TSM_F16, x.data_ptr(), x.data_ptr() + 16, 1,
                             None) == abi.TSM_ERR_INVALID_ARG
    # aliasing in/out
    assert lib.tsm_dslash_tm(g.handle, 0.1, 0.1, 0, abi.TSM_F32, x.data_ptr(), x.data_ptr(), 1,
                             None) == abi.TSM_ERR_INVALID_ARG
    assert lib.tsm_dslash_tm(g.handle, float("nan"), 0.1, 0, abi.TSM_F32, x.data_ptr(), x.data_ptr() + 16, 1,
                             None) == abi.TSM_ERR_INVALID_ARG
    g.close()


def test_rejects_non_unitary_links(ctx):
    import ctypes
    dims = (2, 2, 2, 2)
    links = synth.gauge_links(dims, 0.3, 1)
    links[0, 0, 0, 1, 2] *= 1.01
    h = ctypes.c_void_p()
    dims_c = (ctypes.c_int * 4)(*dims)
    arr = np.ascontiguousarray(links)
    rc = abi.lib().tsm_create_gauge(ctx.handle, dims_c, arr.ctypes.data_as(ctypes.c_void_p), -1, 1, ctypes.byref(h))
    assert rc == abi.TSM_ERR_INVALID_ARG
    links[0, 0, 0, 1, 2] = np.nan
    arr = np.ascontiguousarray(links)
    rc = abi.lib().tsm_create_gauge(ctx.handle, dims_c, arr.ctypes.data_as(ctypes.c_void_p), -1, 1, ctypes.byref(h))
    assert rc == abi.TSM_ERR_NONFINITE


# The Schur operator is two half-volume hops with a stored intermediate, so
# its 16-bit error budget is twice the single operator's.
TOL_MHAT = {abi.TSM_F64: 1e-13, abi.TSM_F32: 4e-6, abi.TSM_F16: 6e-3, abi.TSM_BF16: 6e-2}


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (8, 6, 4, 10), (2, 4, 2, 2)])
@pytest.mark.parametrize("t_bc", [-1, 1])
@pytest.mark.parametrize("prec", [abi.TSM_F64, abi.TSM_F32, abi.TSM_F16, abi.TSM_BF16])
def test_schur_operator_matches_oracle(ctx, dims, t_bc, prec):
    from oracle import evenodd
    kappa, mu = 0.13, 0.07
    g, links = gauge(ctx, dims, 0.35, 21, t_bc)
    u = lattice.effective_links(links, t_bc)
    psi = round_to(synth.gaussian_spinor(dims, 22, nrhs=2), prec)
    nat = g.pack(to_device(psi), prec)
    for op, fn in ((abi.TSM_OP_MHAT, evenodd.apply_mhat), (abi.TSM_OP_MHATDAG, evenodd.apply_mhat_dag)):
        out = g.unpack(g.dslash(op, kappa, mu, prec, nat, 2), prec, 2).cpu().numpy()
        for r in range(2):
            want = fn(u, psi[r], dims, kappa, mu)
            _check(out[r], want, TOL_MHAT[prec])
            assert np.all(evenodd.restrict(out[r], dims, 0) == 0)
    g.close()


@pytest.mark.parametrize("dims", [(3, 4, 2, 2), (4, 3, 2, 2), (4, 4, 2, 3)])
def test_schur_operator_rejects_odd_extents(ctx, dims):
    g, _ = gauge(ctx, dims, 0.3, 1, -1, precs=(abi.TSM_F64,))
    nat = g.pack(to_device(synth.gaussian_spinor(dims, 1, nrhs=1)), abi.TSM_F64)
    with pytest.raises(abi.TsmError):
        g.dslash(abi.TSM_OP_MHAT, 0.1, 0.1, abi.TSM_F64, nat, 1)
    g.close()
