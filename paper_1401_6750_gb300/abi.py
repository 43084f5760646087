"""ctypes binding of the C ABI in include/tsm.h (argument marshalling only).

Every function keeps its C name.  ``lib()`` loads the in-tree shared library
and raises if it has not been built -- there is no fallback.
"""
import ctypes
import os
import re

from . import build as _build

c_int, c_double, c_uint64, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                                 ctypes.c_void_p, ctypes.c_size_t)

TSM_OK, TSM_ERR_INVALID_ARG, TSM_ERR_CUDA, TSM_ERR_OOM = 0, 1, 2, 3
TSM_ERR_NOT_CONVERGED, TSM_ERR_NONFINITE, TSM_ERR_UNIMPLEMENTED = 4, 5, 6
TSM_F64, TSM_F32, TSM_F16, TSM_BF16 = 0, 1, 2, 3
TSM_OP_M, TSM_OP_MDAG, TSM_OP_A, TSM_OP_MDAGM, TSM_OP_MHAT, TSM_OP_MHATDAG = 0, 1, 2, 3, 4, 5
TSM_SOLVER_F64, TSM_SOLVER_F32_RELIABLE, TSM_SOLVER_LP_F16, TSM_SOLVER_LP_BF16 = 0, 1, 2, 3
TSM_SOLVER_EO = 16  # flag: even-odd preconditioned CG (OR with a solver)
TSM_N_INSERTIONS = 160
TSM_CONTRACT_NOALLOC_MAX_BYTES = 32 * 1024 * 1024
CHUNKS = {TSM_F64: 12, TSM_F32: 6, TSM_F16: 3, TSM_BF16: 3}


def prec_bit(p):
    return 1 << p


class tsm_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("reliable_updates", c_int), ("converged", c_int),
                ("restarts", c_int), ("true_residual", c_double)]


class tsm_params(ctypes.Structure):
    _fields_ = [("kappa", c_double), ("mu", c_double), ("n_lp", c_int), ("n_hp", c_int),
                ("rho_lp", c_double), ("rho_hp", c_double), ("lp_solver", c_int), ("hp_solver", c_int),
                ("noise_seed", c_uint64), ("max_iter", c_int), ("nrhs_per_launch", c_int),
                ("n_mom", c_int), ("mom", ctypes.POINTER(c_int))]


class tsm_stats(ctypes.Structure):
    _fields_ = [("lp_iterations_total", c_int), ("hp_iterations_total", c_int),
                ("lp_max_iterations", c_int), ("hp_max_iterations", c_int),
                ("lp_max_true_residual", c_double), ("hp_max_true_residual", c_double),
                ("n_not_converged", c_int), ("seconds", c_double)]


class tsm_batch_item(ctypes.Structure):
    _fields_ = [("gauge", c_void_p), ("kappa", c_double), ("mu", c_double), ("noise_seed", c_uint64),
                ("first_src", c_uint64), ("nsrc", c_int), ("s_dev", c_void_p),
                ("stats_host", ctypes.POINTER(tsm_solve_stats))]


class tsm_kernel_profile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_longlong), ("seconds", c_double),
                ("bytes", c_double), ("flops", c_double)]


_P = c_void_p
_SIGNATURES = {
    "tsm_ctx_create": (c_int, [c_int, ctypes.POINTER(_P)]),
    "tsm_ctx_destroy": (None, [_P]),
    "tsm_create_gauge": (c_int, [_P, ctypes.POINTER(c_int), _P, c_int, ctypes.c_uint, ctypes.POINTER(_P)]),
    "tsm_destroy_gauge": (None, [_P]),
    "tsm_spinor_bytes": (c_size_t, [_P, c_int, c_int]),
    "tsm_spinor_pack": (c_int, [_P, c_int, _P, _P, c_int, c_double, _P]),
    "tsm_spinor_unpack": (c_int, [_P, c_int, _P, _P, c_int, c_double, _P]),
    "tsm_dslash_tm": (c_int, [_P, c_double, c_double, c_int, c_int, _P, _P, c_int, _P]),
    "tsm_make_sources": (c_int, [_P, c_uint64, c_uint64, c_int, c_int, _P, _P]),
    "tsm_make_diluted_sources": (c_int, [_P, c_uint64, c_uint64, c_int, c_int, c_int, _P, _P]),
    "tsm_contract_tdil": (c_int, [_P, c_int, _P, _P, c_int, ctypes.POINTER(c_int), c_int, ctypes.POINTER(c_int),
                                  _P, c_int, _P]),
    "tsm_contract_hpe": (c_int, [_P, c_double, c_double, c_int, _P, _P, c_int, ctypes.POINTER(c_int), c_int,
                                 ctypes.POINTER(c_int), _P, c_int, _P]),
    "tsm_generate_gauge_host": (c_int, [ctypes.POINTER(c_int), c_double, c_uint64, ctypes.POINTER(c_double)]),
    "tsm_binstore_open": (c_int, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(c_void_p)]),
    "tsm_binstore_close": (None, [_P]),
    "tsm_binstore_sources": (ctypes.c_longlong, [_P]),
    "tsm_binstore_block": (c_int, [c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "tsm_binstore_put": (c_int, [_P, c_int, ctypes.POINTER(c_double)]),
    "tsm_binstore_mean": (c_int, [_P, ctypes.c_longlong, ctypes.POINTER(c_double)]),
    "tsm_accumulate_blocks": (c_int, [_P, ctypes.POINTER(tsm_params), _P, c_int, ctypes.POINTER(tsm_stats), _P]),
    "tsm_solve_sources": (c_int, [_P, c_double, c_double, c_int, c_double, c_int, c_uint64, c_uint64,
                                  c_int, c_int, _P, ctypes.POINTER(tsm_solve_stats), _P]),
    "tsm_solve_batch": (c_int, [ctypes.POINTER(tsm_batch_item), c_int, c_int, c_double, c_int, _P]),
    "tsm_invert": (c_int, [_P, c_double, c_double, c_int, c_int, c_double, c_int, _P, _P, c_int,
                           ctypes.POINTER(tsm_solve_stats), _P]),
    "tsm_contract_loops": (c_int, [_P, c_double, c_double, c_int, _P, c_int, c_int, ctypes.POINTER(c_int),
                                   _P, c_int, _P]),
    "tsm_loops_backward": (c_int, [_P, c_double, c_double, c_int, _P, c_int, c_int, ctypes.POINTER(c_int), _P,
                                   c_int, c_double, c_int, ctypes.POINTER(c_double), _P, _P]),
    "tsm_contract_loops_noalloc": (c_int, [_P, c_double, c_double, c_int, _P, c_int, c_int,
                                           ctypes.POINTER(c_int), _P, c_int, _P]),
    "tsm_solve_tsm": (c_int, [_P, ctypes.POINTER(tsm_params), _P, _P, ctypes.POINTER(tsm_stats), _P]),
    "tsm_solve_tsm_dev": (c_int, [_P, ctypes.POINTER(tsm_params), _P, _P, ctypes.POINTER(tsm_stats), _P]),
    "tsm_momentum_table": (c_int, [c_int, ctypes.POINTER(c_int), c_int]),
    "tsm_profile_enable": (c_int, [c_int]),
    "tsm_kernel_launches": (ctypes.c_longlong, []),
    "tsm_profile_read": (c_int, [ctypes.POINTER(tsm_kernel_profile), c_int]),
    "tsm_strerror": (ctypes.c_char_p, [c_int]),
    "tsm_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path():
    return _build.library_path()


def lib():
    """Load the CUDA library (raises if it is missing: build it first)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is not built; run paper_1401_6750_gb300.build.build()" % path)
        handle = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def header_functions(header=None):
    """Names of the functions declared in include/tsm.h."""
    if header is None:
        header = os.path.join(_build.INCLUDE, "tsm.h")
    with open(header) as fh:
        text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
    return sorted(set(re.findall(r"\b(tsm_[a-z0-9_]+)\s*\(", text)))


class TsmError(RuntimeError):
    def __init__(self, code, where):
        l = lib()
        msg = "%s: %s (%s)" % (where, l.tsm_strerror(code).decode(), l.tsm_last_error().decode())
        super().__init__(msg)
        self.code = code


def check(code, where, allow=()):
    if code != TSM_OK and code not in allow:
        raise TsmError(code, where)
    return code
