"""PyTorch-facing wrappers: device memory and streams come from torch, every
step of the computation runs in the CUDA library through ``abi``.

Fields cross the boundary as torch tensors: plain spinors are complex128
tensors of shape (nrhs, T, Lz, Ly, Lx, 4, 3); native fields are uint8
tensors holding the chunked layout described in include/tsm.h.
"""
import ctypes

import numpy as np
import torch

from . import abi


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def solution_prec(solver):
    """Native precision of the solutions a solver returns."""
    kind = solver & ~abi.TSM_SOLVER_EO
    return abi.TSM_F64 if kind in (abi.TSM_SOLVER_F64, abi.TSM_SOLVER_F32_RELIABLE) else abi.TSM_F32


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Context:
    def __init__(self, device=0):
        self.device = device
        torch.cuda.set_device(device)
        h = ctypes.c_void_p()
        abi.check(abi.lib().tsm_ctx_create(device, ctypes.byref(h)), "tsm_ctx_create")
        self.handle = h

    def close(self):
        if self.handle:
            abi.lib().tsm_ctx_destroy(self.handle)
            self.handle = None


class Gauge:
    """Gauge field on the device in the requested precisions."""

    def __init__(self, ctx, links, dims, t_bc=-1, precisions=(abi.TSM_F64, abi.TSM_F32, abi.TSM_F16, abi.TSM_BF16)):
        self.ctx = ctx
        self.dims = tuple(int(d) for d in dims)
        lx, ly, lz, lt = self.dims
        self.volume = lx * ly * lz * lt
        self.t_bc = t_bc
        arr = np.ascontiguousarray(links, dtype=np.complex128)
        assert arr.size == self.volume * 36, "links must hold V*4*3*3 complex numbers"
        mask = 0
        for p in precisions:
            mask |= abi.prec_bit(p)
        h = ctypes.c_void_p()
        dims_c = (ctypes.c_int * 4)(*self.dims)
        abi.check(abi.lib().tsm_create_gauge(ctx.handle, dims_c, arr.ctypes.data_as(ctypes.c_void_p), t_bc, mask,
                                             ctypes.byref(h)), "tsm_create_gauge")
        self.handle = h

    def close(self):
        if self.handle:
            abi.lib().tsm_destroy_gauge(self.handle)
            self.handle = None

    # ---------------------------------------------------------------- fields
    def field_shape(self, nrhs):
        lx, ly, lz, lt = self.dims
        return (nrhs, lt, lz, ly, lx, 4, 3)

    def native_bytes(self, prec, nrhs):
        return int(abi.lib().tsm_spinor_bytes(self.handle, prec, nrhs))

    def empty_native(self, prec, nrhs):
        return torch.empty(self.native_bytes(prec, nrhs), dtype=torch.uint8, device="cuda")

    def pack(self, plain, prec, scale=1.0, stream=None):
        plain = plain.to(device="cuda", dtype=torch.complex128).contiguous()
        nrhs = plain.shape[0]
        out = self.empty_native(prec, nrhs)
        abi.check(abi.lib().tsm_spinor_pack(self.handle, prec, _ptr(plain), _ptr(out), nrhs, scale, _stream(stream)),
                  "tsm_spinor_pack")
        return out

    def unpack(self, native, prec, nrhs, scale=1.0, stream=None):
        out = torch.empty(self.field_shape(nrhs), dtype=torch.complex128, device="cuda")
        abi.check(abi.lib().tsm_spinor_unpack(self.handle, prec, _ptr(native), _ptr(out), nrhs, scale,
                                              _stream(stream)), "tsm_spinor_unpack")
        return out

    # ---------------------------------------------------------------- operators
    def dslash(self, op, kappa, mu, prec, native_in, nrhs, out=None, stream=None):
        if out is None:
            out = self.empty_native(prec, nrhs)
        abi.check(abi.lib().tsm_dslash_tm(self.handle, kappa, mu, op, prec, _ptr(native_in), _ptr(out), nrhs,
                                          _stream(stream)), "tsm_dslash_tm")
        return out

    def sources(self, noise_seed, first_src, nsrc, prec, stream=None):
        out = self.empty_native(prec, nsrc)
        abi.check(abi.lib().tsm_make_sources(self.handle, noise_seed, first_src, nsrc, prec, _ptr(out),
                                             _stream(stream)), "tsm_make_sources")
        return out

    def solve_sources(self, kappa, mu, solver, rho, noise_seed, first_src, nsrc, max_iter=100000, nrhs_per_launch=0,
                      out=None, stream=None, allow_not_converged=False):
        prec = solution_prec(solver)
        if out is None:
            out = self.empty_native(prec, nsrc)
        stats = (abi.tsm_solve_stats * nsrc)()
        rc = abi.lib().tsm_solve_sources(self.handle, kappa, mu, solver, rho, max_iter, noise_seed, first_src, nsrc,
                                         nrhs_per_launch, _ptr(out), stats, _stream(stream))
        allow = (abi.TSM_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        abi.check(rc, "tsm_solve_sources", allow)
        return out, [dict((f, getattr(s, f)) for f, _ in s._fields_) for s in stats]

    def invert(self, op, kappa, mu, solver, rho, native_b, nrhs, max_iter=100000, out=None, stream=None):
        prec = solution_prec(solver)
        if out is None:
            out = self.empty_native(prec, nrhs)
        stats = (abi.tsm_solve_stats * nrhs)()
        abi.check(abi.lib().tsm_invert(self.handle, kappa, mu, op, solver, rho, max_iter, _ptr(native_b), _ptr(out),
                                       nrhs, stats, _stream(stream)), "tsm_invert")
        return out, [dict((f, getattr(s, f)) for f, _ in s._fields_) for s in stats]

    def contract(self, kappa, mu, prec, native_s, nsrc, moms, out=None, accumulate=False, stream=None):
        moms = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1, 3))
        n_mom = moms.shape[0]
        if out is None:
            out = torch.zeros((abi.TSM_N_INSERTIONS, n_mom, self.dims[3], 2), dtype=torch.float64, device="cuda")
        mom_c = moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        abi.check(abi.lib().tsm_contract_loops(self.handle, kappa, mu, prec, _ptr(native_s), nsrc, n_mom, mom_c,
                                               _ptr(out), int(accumulate), _stream(stream)), "tsm_contract_loops")
        return out

    def diluted_sources(self, noise_seed, source_id, t_first, n_t, prec, stream=None):
        """Time dilution: the Z4 source (noise_seed, source_id) on timeslices
        t_first .. t_first + n_t - 1, one field each."""
        out = self.empty_native(prec, n_t)
        abi.check(abi.lib().tsm_make_diluted_sources(self.handle, noise_seed, source_id, t_first, n_t, prec,
                                                     _ptr(out), _stream(stream)), "tsm_make_diluted_sources")
        return out

    def contract_tdil(self, prec, native_s, native_eta, nsrc, t0, moms, out=None, accumulate=False, stream=None):
        """Standard-estimator loops (summed over the sources) of sources eta with
        timeslices t0 (-1: volume source) and their solutions s."""
        moms = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1, 3))
        n_mom = moms.shape[0]
        if out is None:
            out = torch.zeros((abi.TSM_N_INSERTIONS, n_mom, self.dims[3], 2), dtype=torch.float64, device="cuda")
        t0_c = None
        if t0 is not None:
            t0_a = np.ascontiguousarray(np.asarray(t0, dtype=np.int32))
            t0_c = t0_a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        abi.check(abi.lib().tsm_contract_tdil(self.handle, prec, _ptr(native_s), _ptr(native_eta), nsrc, t0_c, n_mom,
                                              moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(out),
                                              int(accumulate), _stream(stream)), "tsm_contract_tdil")
        return out

    def contract_hpe(self, kappa, mu, prec, native_s, native_eta, nsrc, t0, moms, out=None, accumulate=False,
                     stream=None):
        """contract_tdil with the hopping parameter expansion of the ultra-local insertions."""
        moms = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1, 3))
        n_mom = moms.shape[0]
        if out is None:
            out = torch.zeros((abi.TSM_N_INSERTIONS, n_mom, self.dims[3], 2), dtype=torch.float64, device="cuda")
        t0_c = None
        if t0 is not None:
            t0_a = np.ascontiguousarray(np.asarray(t0, dtype=np.int32))
            t0_c = t0_a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        abi.check(abi.lib().tsm_contract_hpe(self.handle, kappa, mu, prec, _ptr(native_s), _ptr(native_eta), nsrc,
                                             t0_c, n_mom, moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                             _ptr(out), int(accumulate), _stream(stream)), "tsm_contract_hpe")
        return out

    def tsm(self, kappa, mu, n_lp, n_hp, rho_lp, rho_hp, lp_solver, hp_solver, noise_seed, moms, max_iter=100000,
            nrhs_per_launch=12, want_parts=False, stream=None):
        moms = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1, 3))
        n_mom = moms.shape[0]
        p = abi.tsm_params(kappa, mu, n_lp, n_hp, rho_lp, rho_hp, lp_solver, hp_solver, noise_seed, max_iter,
                           nrhs_per_launch, n_mom, moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        loops = np.zeros((abi.TSM_N_INSERTIONS, n_mom, self.dims[3], 2))
        parts = np.zeros((3, abi.TSM_N_INSERTIONS, n_mom, self.dims[3], 2)) if want_parts else None
        st = abi.tsm_stats()
        rc = abi.lib().tsm_solve_tsm(self.handle, ctypes.byref(p), loops.ctypes.data_as(ctypes.c_void_p),
                                     parts.ctypes.data_as(ctypes.c_void_p) if want_parts else None,
                                     ctypes.byref(st), _stream(stream))
        abi.check(rc, "tsm_solve_tsm")
        stats = dict((f, getattr(st, f)) for f, _ in st._fields_)
        out = loops[..., 0] + 1j * loops[..., 1]
        if want_parts:
            return out, parts[..., 0] + 1j * parts[..., 1], stats
        return out, stats


def solve_batch(instances, solver, rho, max_iter=100000, stream=None, allow_not_converged=False):
    """Uneven batch in one launch per CG kernel.  instances: list of dicts with
    keys gauge, kappa, mu, noise_seed, first_src, nsrc.  Returns a list of
    (solutions native tensor, stats list) per instance."""
    n = len(instances)
    items = (abi.tsm_batch_item * n)()
    outs, stats = [], []
    for k, inst in enumerate(instances):
        g = inst["gauge"]
        out = g.empty_native(solution_prec(solver), inst["nsrc"])
        st = (abi.tsm_solve_stats * inst["nsrc"])()
        items[k] = abi.tsm_batch_item(g.handle.value, inst["kappa"], inst["mu"], inst["noise_seed"],
                                      inst["first_src"], inst["nsrc"], out.data_ptr(),
                                      ctypes.cast(st, ctypes.POINTER(abi.tsm_solve_stats)))
        outs.append(out)
        stats.append(st)
    rc = abi.lib().tsm_solve_batch(items, n, solver, rho, max_iter, _stream(stream))
    abi.check(rc, "tsm_solve_batch", (abi.TSM_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return [(o, [dict((f, getattr(x, f)) for f, _ in x._fields_) for x in st]) for o, st in zip(outs, stats)]


def momentum_table(p2max=9):
    n = abi.lib().tsm_momentum_table(p2max, None, 0)
    buf = (ctypes.c_int * (3 * n))()
    abi.lib().tsm_momentum_table(p2max, buf, n)
    return [tuple(buf[3 * k:3 * k + 3]) for k in range(n)]


def loops_complex(out):
    """[160][n_mom][T][2] float64 tensor -> complex128 numpy array."""
    a = out.detach().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


class OneEndLoops(torch.autograd.Function):
    """Differentiable one-end loops (Sec. 2.1.1) of caller sources.

    forward(mu, eta): s = M(mu)^{-1} eta by `solver` (tsm_invert), loops of
    all 160 insertions on `moms` summed over the sources (tsm_contract_loops,
    in `prec`), returned as complex128 (160, n_mom, T).
    backward: tsm_loops_backward (adjoint solve with M^dag) -> dl/dmu and
    dl/deta.  mu is a 0-d float64 tensor, eta complex128 (nsrc, T, Lz, Ly, Lx, 4, 3).
    """

    @staticmethod
    def forward(ctx, mu, eta, gauge, kappa, moms, solver, rho, prec, max_iter):
        mu_v = float(mu)
        nsrc = eta.shape[0]
        b = gauge.pack(eta.detach(), solution_prec(solver))
        s, _ = gauge.invert(abi.TSM_OP_M, kappa, mu_v, solver, rho, b, nsrc, max_iter=max_iter)
        if prec != solution_prec(solver):
            s = gauge.pack(gauge.unpack(s, solution_prec(solver), nsrc), prec)
        out = gauge.contract(kappa, mu_v, prec, s, nsrc, moms)
        ctx.gauge, ctx.kappa, ctx.mu, ctx.solver, ctx.rho, ctx.prec = gauge, kappa, mu_v, solver, rho, prec
        ctx.max_iter, ctx.nsrc, ctx.s = max_iter, nsrc, s
        ctx.moms = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1, 3))
        ctx.mu_meta = (mu.dtype, mu.device)
        ctx.eta_meta = (eta.dtype, eta.device)
        return torch.view_as_complex(out.contiguous())

    @staticmethod
    def backward(ctx, grad_loops):
        g = ctx.gauge
        gd = torch.view_as_real(grad_loops.to(device="cuda", dtype=torch.complex128).contiguous()).contiguous()
        dmu = ctypes.c_double()
        grad_eta = g.empty_native(ctx.prec, ctx.nsrc) if ctx.needs_input_grad[1] else None
        mom_c = ctx.moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        abi.check(abi.lib().tsm_loops_backward(g.handle, ctx.kappa, ctx.mu, ctx.prec, _ptr(ctx.s), ctx.nsrc,
                                               ctx.moms.shape[0], mom_c, _ptr(gd), ctx.solver, ctx.rho,
                                               ctx.max_iter, ctypes.byref(dmu),
                                               _ptr(grad_eta) if grad_eta is not None else None, _stream()),
                  "tsm_loops_backward")
        dmu_t = torch.tensor(dmu.value, dtype=ctx.mu_meta[0], device=ctx.mu_meta[1])
        geta = None
        if grad_eta is not None:
            geta = g.unpack(grad_eta, ctx.prec, ctx.nsrc).to(dtype=ctx.eta_meta[0], device=ctx.eta_meta[1])
        return dmu_t, geta, None, None, None, None, None, None, None


def one_end_loops(mu, eta, gauge, kappa, moms, solver=abi.TSM_SOLVER_F64, rho=1e-12, prec=abi.TSM_F64,
                  max_iter=100000):
    return OneEndLoops.apply(mu, eta, gauge, kappa, moms, solver, rho, prec, max_iter)


class BinStore:
    """Binary-weight storage of loop sums (block k: sources 2^k - 1 ..
    2^{k+1} - 2, any N from its bits).  Host-side; `accumulate` fills it on
    the GPU with the bulk LP loops."""

    def __init__(self, path_prefix, n_values):
        self.n_values = int(n_values)
        h = ctypes.c_void_p()
        abi.check(abi.lib().tsm_binstore_open(str(path_prefix).encode(), self.n_values, ctypes.byref(h)),
                  "tsm_binstore_open")
        self.handle = h

    def close(self):
        if self.handle:
            abi.lib().tsm_binstore_close(self.handle)
            self.handle = None

    @property
    def sources(self):
        return int(abi.lib().tsm_binstore_sources(self.handle))

    @staticmethod
    def block(k):
        first, count = ctypes.c_longlong(), ctypes.c_longlong()
        abi.check(abi.lib().tsm_binstore_block(k, ctypes.byref(first), ctypes.byref(count)), "tsm_binstore_block")
        return first.value, count.value

    def put(self, k, block_sum):
        a = np.ascontiguousarray(np.asarray(block_sum, dtype=np.float64).ravel())
        if a.size != self.n_values:
            raise ValueError("block holds %d values, store expects %d" % (a.size, self.n_values))
        abi.check(abi.lib().tsm_binstore_put(self.handle, k, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                  "tsm_binstore_put")

    def mean(self, n):
        out = np.empty(self.n_values, dtype=np.float64)
        abi.check(abi.lib().tsm_binstore_mean(self.handle, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                  "tsm_binstore_mean")
        return out

    def accumulate(self, gauge, kappa, mu, lp_solver, rho_lp, noise_seed, moms, k_end, max_iter=100000,
                   nrhs_per_launch=32, stream=None):
        moms = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1, 3))
        p = abi.tsm_params(kappa, mu, 0, 0, rho_lp, 0.5, lp_solver, lp_solver, noise_seed, max_iter,
                           nrhs_per_launch, moms.shape[0], moms.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        st = abi.tsm_stats()
        abi.check(abi.lib().tsm_accumulate_blocks(gauge.handle, ctypes.byref(p), self.handle, k_end,
                                                  ctypes.byref(st), _stream(stream)), "tsm_accumulate_blocks")
        return dict((f, getattr(st, f)) for f, _ in st._fields_)


def generate_gauge_host(dims, eps, seed):
    """The library's host generator of U = exp(i eps H) links (see
    tsm_generate_gauge_host): complex128 (T, Lz, Ly, Lx, 4, 3, 3)."""
    lx, ly, lz, lt = dims
    out = np.empty((lt, lz, ly, lx, 4, 3, 3, 2), dtype=np.float64)
    d = (ctypes.c_int * 4)(*dims)
    abi.check(abi.lib().tsm_generate_gauge_host(d, eps, seed, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
              "tsm_generate_gauge_host")
    return out[..., 0] + 1j * out[..., 1]
