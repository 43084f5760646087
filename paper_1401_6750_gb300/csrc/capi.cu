// extern "C" entry points declared in include/tsm.h: argument checks, device
// binding and dispatch to the launchers.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace tsm {

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  cudaGetLastError();  // clear a non-sticky error
  const int code = (e == cudaErrorMemoryAllocation) ? TSM_ERR_OOM : TSM_ERR_CUDA;
  return fail(code, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

int DevBuf::reserve(size_t n) {
  if (n <= bytes && p) return TSM_OK;
  release();
  if (n == 0) n = 16;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    return cuda_status(e, "cudaMalloc", __FILE__, __LINE__);
  }
  bytes = n;
  return TSM_OK;
}

int UseOrder::enter(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TSM_CUDA(cudaStreamIsCapturing(st, &cs));
  capturing = (cs != cudaStreamCaptureStatusNone);
  if (capturing) return TSM_OK;
  if (!done) TSM_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
  TSM_CUDA(cudaStreamWaitEvent(st, done, 0));
  return TSM_OK;
}

int UseOrder::leave(cudaStream_t st) {
  if (capturing || !done) return TSM_OK;
  TSM_CUDA(cudaEventRecord(done, st));
  return TSM_OK;
}

int UseOrder::wait_host() {
  if (done) TSM_CUDA(cudaEventSynchronize(done));
  return TSM_OK;
}

int momentum_table(int p2max, std::vector<int>& out) {
  out.clear();
  if (p2max < 0) return -1;
  int r = 0;
  while ((r + 1) * (r + 1) <= p2max) ++r;
  struct M {
    int n2, x, y, z;
  };
  std::vector<M> v;
  for (int x = -r; x <= r; ++x)
    for (int y = -r; y <= r; ++y)
      for (int z = -r; z <= r; ++z) {
        const int n2 = x * x + y * y + z * z;
        if (n2 <= p2max) v.push_back(M{n2, x, y, z});
      }
  std::sort(v.begin(), v.end(), [](const M& a, const M& b) {
    if (a.n2 != b.n2) return a.n2 < b.n2;
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
  });
  for (const M& m : v) {
    out.push_back(m.x);
    out.push_back(m.y);
    out.push_back(m.z);
  }
  return (int)v.size();
}

static bool valid_prec(int p) { return p >= TSM_F64 && p <= TSM_BF16; }

// Bind the calling host thread to the handle's device.
static int bind(const tsm_gauge* g) {
  TSM_CUDA(cudaSetDevice(g->ctx->device));
  return TSM_OK;
}

}  // namespace tsm

tsm_gauge::~tsm_gauge() {
  if (aux_stream) cudaStreamDestroy(aux_stream);
  for (cudaEvent_t e : aux_ev)
    if (e) cudaEventDestroy(e);
}

using namespace tsm;

extern "C" {

const char* tsm_strerror(int code) {
  switch (code) {
    case TSM_OK: return "ok";
    case TSM_ERR_INVALID_ARG: return "invalid argument";
    case TSM_ERR_CUDA: return "CUDA error";
    case TSM_ERR_OOM: return "out of device memory";
    case TSM_ERR_NOT_CONVERGED: return "solver did not converge";
    case TSM_ERR_NONFINITE: return "non-finite value";
    case TSM_ERR_UNIMPLEMENTED: return "not implemented";
  }
  return "unknown status";
}

const char* tsm_last_error(void) { return g_last_error.c_str(); }

int tsm_ctx_create(int device, tsm_ctx** out) {
  if (!out) return fail(TSM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int n = 0;
  TSM_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(TSM_ERR_INVALID_ARG, "device %d of %d", device, n);
  TSM_CUDA(cudaSetDevice(device));
  cudaDeviceProp prop;
  TSM_CUDA(cudaGetDeviceProperties(&prop, device));
  if (prop.major != 10 || prop.minor != 3)
    return fail(TSM_ERR_CUDA, "library is built for sm_103 only; device %d is sm_%d%d", device, prop.major,
                prop.minor);
  tsm_ctx* c = new tsm_ctx();
  c->device = device;
  c->sm_count = prop.multiProcessorCount;
  cudaError_t e = cudaStreamCreate(&c->stream);
  if (e != cudaSuccess) {
    delete c;
    return cuda_status(e, "cudaStreamCreate", __FILE__, __LINE__);
  }
  *out = c;
  return TSM_OK;
}

void tsm_ctx_destroy(tsm_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

int tsm_create_gauge(tsm_ctx* ctx, const int dims[4], const double* links_host, int t_bc, unsigned precisions,
                     tsm_gauge** out) {
  if (!out) return fail(TSM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ctx || !dims || !links_host) return fail(TSM_ERR_INVALID_ARG, "NULL ctx, dims or links");
  if (t_bc != 1 && t_bc != -1) return fail(TSM_ERR_INVALID_ARG, "t_bc must be +1 or -1, got %d", t_bc);
  if (precisions == 0 || (precisions & ~0xFu)) return fail(TSM_ERR_INVALID_ARG, "bad precision mask 0x%x", precisions);
  long long v = 1;
  for (int d = 0; d < 4; ++d) {
    if (dims[d] < 2 || dims[d] > 4096) return fail(TSM_ERR_INVALID_ARG, "dims[%d] = %d outside [2, 4096]", d, dims[d]);
    v *= dims[d];
  }
  if (v > (1LL << 28)) return fail(TSM_ERR_INVALID_ARG, "volume %lld too large", v);
  // the links must be finite SU(3) matrices (the 12-real copies rebuild row 3)
  for (long long k = 0; k < v * 4; ++k) {
    const double* u = links_host + k * 18;
    for (int c = 0; c < 18; ++c)
      if (!isfinite(u[c])) return fail(TSM_ERR_NONFINITE, "link %lld is not finite", k);
    double dev = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double re = 0, im = 0;
        for (int c = 0; c < 3; ++c) {  // (U U^dag)_ab
          const double ar = u[(a * 3 + c) * 2], ai = u[(a * 3 + c) * 2 + 1];
          const double br = u[(b * 3 + c) * 2], bi = u[(b * 3 + c) * 2 + 1];
          re += ar * br + ai * bi;
          im += ai * br - ar * bi;
        }
        dev = std::max(dev, fabs(re - (a == b ? 1.0 : 0.0)) + fabs(im));
      }
    if (!(dev < 1e-6)) return fail(TSM_ERR_INVALID_ARG, "link %lld is not unitary (|UU^dag - 1| = %g)", k, dev);
  }
  TSM_CUDA(cudaSetDevice(ctx->device));
  tsm_gauge* g = new tsm_gauge();
  g->ctx = ctx;
  for (int d = 0; d < 4; ++d) g->geom.L[d] = dims[d];
  g->geom.V = (int)v;
  g->geom.bc = t_bc;
  for (int d = 0; d < 3; ++d) g->geom.div[d] = make_fastdiv((uint32_t)dims[d]);
  g->precisions = precisions;
  int rc = build_links(g, links_host);
  if (rc != TSM_OK) {
    delete g;
    return rc;
  }
  *out = g;
  return TSM_OK;
}

void tsm_destroy_gauge(tsm_gauge* g) {
  if (!g) return;
  cudaSetDevice(g->ctx->device);
  cudaDeviceSynchronize();
  delete g;
}

size_t tsm_spinor_bytes(const tsm_gauge* g, int prec, int nrhs) {
  if (!g || !valid_prec(prec) || nrhs < 0) return 0;
  return (size_t)nrhs * spinor_chunks(prec) * (size_t)g->geom.V * 16;
}

int tsm_spinor_pack(const tsm_gauge* g, int prec, const double* plain_dev, void* native_dev, int nrhs, double scale,
                    void* stream) {
  if (!g || !plain_dev || !native_dev || !valid_prec(prec) || nrhs < 0)
    return fail(TSM_ERR_INVALID_ARG, "tsm_spinor_pack: bad argument");
  if (nrhs == 0) return TSM_OK;
  TSM_TRY(bind(g));
  return spinor_pack(g, prec, plain_dev, native_dev, nrhs, scale, pick_stream(g, stream));
}

int tsm_spinor_unpack(const tsm_gauge* g, int prec, const void* native_dev, double* plain_dev, int nrhs,
                      double scale, void* stream) {
  if (!g || !plain_dev || !native_dev || !valid_prec(prec) || nrhs < 0)
    return fail(TSM_ERR_INVALID_ARG, "tsm_spinor_unpack: bad argument");
  if (nrhs == 0) return TSM_OK;
  TSM_TRY(bind(g));
  return spinor_unpack(g, prec, native_dev, plain_dev, nrhs, scale, pick_stream(g, stream));
}

int tsm_dslash_tm(tsm_gauge* g, double kappa, double mu, int op, int prec, const void* in_dev, void* out_dev,
                  int nrhs, void* stream) {
  if (!g || !in_dev || !out_dev || !valid_prec(prec) || nrhs < 0 || op < TSM_OP_M || op > TSM_OP_MHATDAG)
    return fail(TSM_ERR_INVALID_ARG, "tsm_dslash_tm: bad argument");
  if (!isfinite(kappa) || !isfinite(mu)) return fail(TSM_ERR_INVALID_ARG, "kappa and mu must be finite");
  if (!has_prec(g, prec)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", prec);
  if (in_dev == out_dev) return fail(TSM_ERR_INVALID_ARG, "in and out must not alias");
  if (nrhs == 0) return TSM_OK;
  if (nrhs > 65535) return fail(TSM_ERR_INVALID_ARG, "nrhs %d > 65535", nrhs);
  TSM_TRY(bind(g));
  if (op == TSM_OP_MHAT || op == TSM_OP_MHATDAG)
    return schur_apply(g, prec, op == TSM_OP_MHATDAG, kappa, mu, in_dev, out_dev, nrhs, pick_stream(g, stream));
  return dslash_apply(g, prec, op, kappa, mu, in_dev, out_dev, nrhs, pick_stream(g, stream));
}

int tsm_make_sources(tsm_gauge* g, uint64_t noise_seed, uint64_t first_src, int nsrc, int prec, void* out_dev,
                     void* stream) {
  if (!g || !out_dev || !valid_prec(prec) || nsrc < 0 || nsrc > 65535)
    return fail(TSM_ERR_INVALID_ARG, "tsm_make_sources: bad argument");
  if (nsrc == 0) return TSM_OK;
  TSM_TRY(bind(g));
  return make_sources(g, noise_seed, first_src, nsrc, prec, out_dev, pick_stream(g, stream));
}

int tsm_generate_gauge_host(const int dims[4], double eps, uint64_t seed, double* links_out) {
  if (!dims || !links_out || !isfinite(eps)) return fail(TSM_ERR_INVALID_ARG, "tsm_generate_gauge_host: bad argument");
  for (int d = 0; d < 4; ++d)
    if (dims[d] < 1) return fail(TSM_ERR_INVALID_ARG, "extent %d is %d", d, dims[d]);
  return generate_gauge_host(dims, eps, seed, links_out);
}

int tsm_make_diluted_sources(tsm_gauge* g, uint64_t noise_seed, uint64_t source_id, int t_first, int n_t, int prec,
                             void* out_dev, void* stream) {
  if (!g || !out_dev || !valid_prec(prec) || n_t < 0 || n_t > 65535 || t_first < 0 ||
      t_first + n_t > g->geom.L[3])
    return fail(TSM_ERR_INVALID_ARG, "tsm_make_diluted_sources: bad argument");
  if (n_t == 0) return TSM_OK;
  TSM_TRY(bind(g));
  return make_diluted_sources(g, noise_seed, source_id, t_first, n_t, prec, out_dev, pick_stream(g, stream));
}

int tsm_contract_tdil(tsm_gauge* g, int prec, const void* s_dev, const void* eta_dev, int nsrc, const int* t0_host,
                      int n_mom, const int* mom, double* out_dev, int accumulate, void* stream) {
  if (!g || !s_dev || !eta_dev || !out_dev || nsrc < 0 || nsrc > 65535 || n_mom < 1 || n_mom > 4096 || !mom)
    return fail(TSM_ERR_INVALID_ARG, "tsm_contract_tdil: bad argument");
  if (nsrc == 0 && accumulate) return TSM_OK;
  TSM_TRY(bind(g));
  return contract_tdil(g, prec, s_dev, eta_dev, nsrc, t0_host, n_mom, mom, out_dev, accumulate,
                       pick_stream(g, stream));
}

int tsm_contract_hpe(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, const void* eta_dev,
                     int nsrc, const int* t0_host, int n_mom, const int* mom, double* out_dev, int accumulate,
                     void* stream) {
  if (!g || !s_dev || !eta_dev || !out_dev || nsrc < 1 || nsrc > 65535 || n_mom < 1 || n_mom > 4096 || !mom)
    return fail(TSM_ERR_INVALID_ARG, "tsm_contract_hpe: bad argument");
  if (!isfinite(kappa) || !isfinite(mu) || kappa <= 0.0) return fail(TSM_ERR_INVALID_ARG, "bad kappa or mu");
  TSM_TRY(bind(g));
  return contract_hpe(g, kappa, mu, prec, s_dev, eta_dev, nsrc, t0_host, n_mom, mom, out_dev, accumulate,
                      pick_stream(g, stream));
}

static int check_solver_args(const tsm_gauge* g, double kappa, double mu, int solver, double rho, int max_iter) {
  if (!g) return fail(TSM_ERR_INVALID_ARG, "gauge is NULL");
  if (solver_kind(solver) < 0) return fail(TSM_ERR_INVALID_ARG, "bad solver %d", solver);
  if ((solver & TSM_SOLVER_EO) && !eo_lattice(g->geom))
    return fail(TSM_ERR_INVALID_ARG, "even-odd solves need even extents in all four directions");
  if (!(rho > 0.0) || !(rho < 1.0)) return fail(TSM_ERR_INVALID_ARG, "rho must lie in (0, 1), got %g", rho);
  if (max_iter < 1) return fail(TSM_ERR_INVALID_ARG, "max_iter must be >= 1");
  if (!isfinite(kappa) || !isfinite(mu) || kappa <= 0.0) return fail(TSM_ERR_INVALID_ARG, "bad kappa or mu");
  const unsigned need = solver_link_precs(solver);
  if ((g->precisions & need) != need)
    return fail(TSM_ERR_INVALID_ARG, "solver %d needs gauge copies 0x%x, gauge has 0x%x", solver, need, g->precisions);
  return TSM_OK;
}

int tsm_solve_sources(tsm_gauge* g, double kappa, double mu, int solver, double rho, int max_iter,
                      uint64_t noise_seed, uint64_t first_src, int nsrc, int nrhs_per_launch, void* s_dev,
                      tsm_solve_stats* stats_host, void* stream) {
  TSM_TRY(check_solver_args(g, kappa, mu, solver, rho, max_iter));
  if (!s_dev || nsrc < 0) return fail(TSM_ERR_INVALID_ARG, "tsm_solve_sources: bad output or count");
  if (nsrc == 0) return TSM_OK;
  TSM_TRY(bind(g));
  cudaStream_t s = pick_stream(g, stream);
  const int batch = (nrhs_per_launch <= 0) ? nsrc : std::min(nrhs_per_launch, nsrc);
  if (batch > 1024) return fail(TSM_ERR_INVALID_ARG, "at most 1024 right-hand sides per launch");
  const int op = solver_output_prec(solver);
  const size_t field = tsm_spinor_bytes(g, op, 1);
  int worst = TSM_OK;
  for (int k0 = 0; k0 < nsrc; k0 += batch) {
    const int n = std::min(batch, nsrc - k0);
    int rc = solve_batch_impl(g, kappa, mu, solver, rho, max_iter, n, nullptr, 0, noise_seed, first_src + k0, op,
                              static_cast<char*>(s_dev) + field * k0, 0, stats_host ? stats_host + k0 : nullptr, s);
    if (rc == TSM_ERR_NOT_CONVERGED) {
      worst = rc;
      continue;
    }
    if (rc != TSM_OK) return rc;
  }
  if (worst != TSM_OK) return fail(worst, "some sources did not reach rho");
  return TSM_OK;
}

int tsm_solve_batch(tsm_batch_item* items, int n_items, int solver, double rho, int max_iter, void* stream) {
  if (!items || n_items < 1 || n_items > 64) return fail(TSM_ERR_INVALID_ARG, "need 1 to 64 batch items");
  if (solver & TSM_SOLVER_EO) return fail(TSM_ERR_INVALID_ARG, "tsm_solve_batch has no even-odd variant");
  long long rhs = 0;
  for (int k = 0; k < n_items; ++k) {
    const tsm_batch_item& it = items[k];
    TSM_TRY(check_solver_args(it.gauge, it.kappa, it.mu, solver, rho, max_iter));
    if (!it.s_dev || it.nsrc < 1 || it.nsrc > 1024) return fail(TSM_ERR_INVALID_ARG, "item %d: bad output or count", k);
    if (it.gauge->ctx->device != items[0].gauge->ctx->device)
      return fail(TSM_ERR_INVALID_ARG, "item %d lives on another device", k);
    rhs += it.nsrc;
  }
  if (rhs > 65536) return fail(TSM_ERR_INVALID_ARG, "at most 65536 right-hand sides per batch");
  TSM_TRY(bind(items[0].gauge));
  return solve_batch_multi(items, n_items, solver, rho, max_iter, pick_stream(items[0].gauge, stream));
}

int tsm_invert(tsm_gauge* g, double kappa, double mu, int op, int solver, double rho, int max_iter,
               const void* b_dev, void* x_dev, int nrhs, tsm_solve_stats* stats_host, void* stream) {
  TSM_TRY(check_solver_args(g, kappa, mu, solver, rho, max_iter));
  if (!b_dev || !x_dev || nrhs < 0 || (op != TSM_OP_M && op != TSM_OP_MDAG))
    return fail(TSM_ERR_INVALID_ARG, "tsm_invert: bad argument");
  if (nrhs == 0) return TSM_OK;
  if (nrhs > 1024) return fail(TSM_ERR_INVALID_ARG, "at most 1024 right-hand sides");
  TSM_TRY(bind(g));
  const int p = solver_output_prec(solver);
  // M^dag x = b  <=>  M(-mu) (g5 x) = g5 b
  const int dag = (op == TSM_OP_MDAG);
  return solve_batch_impl(g, kappa, dag ? -mu : mu, solver, rho, max_iter, nrhs, b_dev, p, 0, 0, p, x_dev, dag,
                          stats_host, pick_stream(g, stream));
}

int tsm_contract_loops(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                       const int* mom, double* out_dev, int accumulate, void* stream) {
  if (!g || !s_dev || !out_dev || nsrc < 0 || n_mom < 1 || !mom)
    return fail(TSM_ERR_INVALID_ARG, "tsm_contract_loops: bad argument");
  if (nsrc > 65535) return fail(TSM_ERR_INVALID_ARG, "nsrc %d > 65535", nsrc);
  if (!isfinite(kappa) || !isfinite(mu)) return fail(TSM_ERR_INVALID_ARG, "kappa and mu must be finite");
  TSM_TRY(bind(g));
  cudaStream_t s = pick_stream(g, stream);
  if (nsrc == 0) {
    if (!accumulate)
      TSM_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double) * 2 * 160 * (size_t)n_mom * g->geom.L[3], s));
    return TSM_OK;
  }
  return contract_loops(g, kappa, mu, prec, s_dev, nsrc, n_mom, mom, out_dev, accumulate, s);
}

int tsm_contract_loops_noalloc(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc,
                               int n_mom, const int* mom, double* out_dev, int accumulate, void* stream) {
  if (!g || !s_dev || !out_dev || nsrc < 0 || n_mom < 1 || !mom)
    return fail(TSM_ERR_INVALID_ARG, "tsm_contract_loops_noalloc: bad argument");
  if (nsrc > 65535) return fail(TSM_ERR_INVALID_ARG, "nsrc %d > 65535", nsrc);
  if (!isfinite(kappa) || !isfinite(mu)) return fail(TSM_ERR_INVALID_ARG, "kappa and mu must be finite");
  TSM_TRY(bind(g));
  cudaStream_t s = pick_stream(g, stream);
  if (nsrc == 0) {
    if (!accumulate)
      TSM_CUDA(cudaMemsetAsync(out_dev, 0, sizeof(double) * 2 * 160 * (size_t)n_mom * g->geom.L[3], s));
    return TSM_OK;
  }
  return contract_loops_noalloc(g, kappa, mu, prec, s_dev, nsrc, n_mom, mom, out_dev, accumulate, s);
}

int tsm_loops_backward(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                       const int* mom, const double* grad_dev, int solver, double rho, int max_iter, double* dmu_host,
                       void* grad_eta_dev, void* stream) {
  if (!g || !s_dev || !grad_dev || !dmu_host || nsrc < 1 || n_mom < 1 || !mom)
    return fail(TSM_ERR_INVALID_ARG, "tsm_loops_backward: bad argument");
  if (prec != TSM_F64 && prec != TSM_F32) return fail(TSM_ERR_INVALID_ARG, "solutions must be F64 or F32");
  if (solver_kind(solver) != TSM_SOLVER_F64 && solver_kind(solver) != TSM_SOLVER_F32_RELIABLE)
    return fail(TSM_ERR_INVALID_ARG, "the adjoint solve needs TSM_SOLVER_F64 or TSM_SOLVER_F32_RELIABLE");
  TSM_TRY(check_solver_args(g, kappa, mu, solver, rho, max_iter));
  if (!has_prec(g, prec)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", prec);
  if (nsrc > 1024) return fail(TSM_ERR_INVALID_ARG, "at most 1024 sources");
  for (int m = 0; m < 3 * n_mom; ++m)
    if (mom[m] > 8 || mom[m] < -8) return fail(TSM_ERR_INVALID_ARG, "momentum component outside [-8, 8]");
  TSM_TRY(bind(g));
  return loops_backward(g, kappa, mu, prec, s_dev, nsrc, n_mom, mom, grad_dev, solver, rho, max_iter, dmu_host,
                        grad_eta_dev, pick_stream(g, stream));
}

int tsm_momentum_table(int p2max, int* out, int cap) {
  std::vector<int> v;
  const int n = momentum_table(p2max, v);
  if (n < 0) {
    fail(TSM_ERR_INVALID_ARG, "p2max must be >= 0");
    return -1;
  }
  if (out)
    for (int k = 0; k < std::min(n, cap) * 3; ++k) out[k] = v[k];
  return n;
}

}  // extern "C"
