"""Allocation-free contraction (tsm_contract_loops_noalloc) against the
regular entry point, through the C ABI.

Some callers cannot allocate device memory while they call the library (an
allocator or memory pool that forbids new device allocations, or a loop that
must not synchronise the device); for them the contraction keeps its scratch
in a fixed array compiled into the library.  This file is collected last so
that a failure here comes after every other test has run; it passes both
alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_helpers import gauge, round_to, to_device
from oracle import momenta
from paper_1401_6750_gb300 import abi, synth

pytestmark = pytest.mark.gpu

TOL = 1e-6  # normwise per insertion, as for the FP32 contraction tests
TOL_F64 = 1e-11  # as for the FP64 contraction tests


def _call(fn, g, kappa, mu, prec, nat, nsrc, moms, out):
    mom = np.ascontiguousarray(np.asarray(moms, dtype=np.int32))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(g.handle, kappa, mu, prec, ctypes.c_void_p(nat.data_ptr()), nsrc, mom.shape[0],
              mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_void_p(out.data_ptr()), 0, stream)


def _loops(out):
    a = out.cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("prec,tol", [(abi.TSM_F32, TOL), (abi.TSM_F64, TOL_F64)])
def test_noalloc_matches_regular_entry_two_calls(ctx, prec, tol):
    dims = (8, 6, 4, 8) if prec == abi.TSM_F32 else (4, 6, 4, 8)
    kappa, mu = 0.125, 0.01
    g, _ = gauge(ctx, dims, 0.3, 7, -1, precs=(prec,))
    lib = abi.lib()
    moms = momenta.momentum_list(9)
    shape = (abi.TSM_N_INSERTIONS, len(moms), dims[3], 2)
    for call, seed in enumerate((70, 71)):  # two calls in a row, different sources
        nsrc = 3 + call
        s = round_to(synth.gaussian_spinor(dims, seed, nrhs=nsrc), prec)
        nat = g.pack(to_device(s), prec)
        ref = torch.full(shape, np.nan, dtype=torch.float64, device="cuda")
        got = torch.full(shape, np.nan, dtype=torch.float64, device="cuda")
        assert _call(lib.tsm_contract_loops, g, kappa, mu, prec, nat, nsrc, moms, ref) == abi.TSM_OK
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free0 = torch.cuda.mem_get_info()[0]
        rc = _call(lib.tsm_contract_loops_noalloc, g, kappa, mu, prec, nat, nsrc, moms, got)
        assert rc == abi.TSM_OK, lib.tsm_last_error()
        torch.cuda.synchronize()
        if call > 0:  # after the first call's one-time set-up the device's free memory is unchanged
            assert torch.cuda.mem_get_info()[0] == free0
        a, b = _loops(got), _loops(ref)
        assert np.all(np.isfinite(a))
        for ins in range(abi.TSM_N_INSERTIONS):
            assert np.linalg.norm(a[ins] - b[ins]) <= tol * np.linalg.norm(b[ins]), (call, ins)
    g.close()


def test_noalloc_rejects_oversize_request(ctx):
    dims = (16, 16, 16, 32)  # the 160 FP32 site fields alone need 160 MiB
    g, _ = gauge(ctx, dims, 0.3, 8, -1, precs=(abi.TSM_F32,))
    lib = abi.lib()
    nat = g.empty_native(abi.TSM_F32, 1)
    out = torch.zeros((abi.TSM_N_INSERTIONS, 123, dims[3], 2), dtype=torch.float64, device="cuda")
    rc = _call(lib.tsm_contract_loops_noalloc, g, 0.125, 0.01, abi.TSM_F32, nat, 1, momenta.momentum_list(9), out)
    assert rc == abi.TSM_ERR_INVALID_ARG
    assert b"scratch" in lib.tsm_last_error()
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0  # output untouched
    g.close()
