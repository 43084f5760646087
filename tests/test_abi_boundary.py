"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/tsm.h declares.  Only host-side helpers are called here."""
import ctypes
import shutil

import pytest

from oracle import momenta
from paper_1401_6750_gb300 import abi, build

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not __import__("os").path.exists(
    "/usr/local/cuda/bin/nvcc"), reason="CUDA toolkit needed to build the library")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return abi.lib()


def test_exports_every_declared_function(lib):
    names = abi.header_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(abi._SIGNATURES) == set(names)


def test_momentum_table_matches_oracle_bit_exact(lib):
    for p2 in (0, 1, 4, 9, 12):
        n = lib.tsm_momentum_table(p2, None, 0)
        buf = (ctypes.c_int * (3 * n))()
        assert lib.tsm_momentum_table(p2, buf, n) == n
        got = [tuple(buf[3 * k:3 * k + 3]) for k in range(n)]
        assert got == momenta.momentum_list(p2)
    assert lib.tsm_momentum_table(-1, None, 0) == -1


def test_error_strings(lib):
    assert lib.tsm_strerror(abi.TSM_OK) == b"ok"
    assert b"converge" in lib.tsm_strerror(abi.TSM_ERR_NOT_CONVERGED)
    assert lib.tsm_strerror(999) == b"unknown status"


def test_invalid_arguments_rejected_before_device_use(lib):
    h = ctypes.c_void_p()
    assert lib.tsm_ctx_create(0, None) == abi.TSM_ERR_INVALID_ARG
    assert lib.tsm_create_gauge(None, None, None, -1, 1, ctypes.byref(h)) == abi.TSM_ERR_INVALID_ARG
    assert lib.tsm_dslash_tm(None, 0.1, 0.1, 0, 0, None, None, 1, None) == abi.TSM_ERR_INVALID_ARG
    assert lib.tsm_solve_tsm(None, None, None, None, None, None) == abi.TSM_ERR_INVALID_ARG
    assert b"NULL" in lib.tsm_last_error() or len(lib.tsm_last_error()) > 0
    assert lib.tsm_spinor_bytes(None, 0, 1) == 0


def test_header_enum_values_match_binding():
    """Every TSM_* enumerator of the header has the value the binding uses."""
    import os
    import re
    text = open(os.path.join(build.INCLUDE, "tsm.h")).read()
    found = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(TSM_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    assert "TSM_SOLVER_EO" in found and "TSM_SOLVER_LP_BF16" in found
    for name, value in found.items():
        if hasattr(abi, name):
            assert getattr(abi, name) == value, name
