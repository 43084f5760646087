// Truncated Solver Method driver (Sec. 2.1) with on-device accumulation of
// the contractions (the "projected scheme" of Fig. 4: sources, inversions,
// contractions, accumulation and the Fourier projection all stay on the GPU;
// only the final estimate crosses to the host).
//
//   E = (1/N_LP) sum_{r < N_LP} L_LP(eta_r)
//     + (1/N_HP) sum_{N_LP <= r < N_LP + N_HP} [ L_HP(eta_r) - L_LP(eta_r) ]
//
// The low-precision map is the same solver call (same precision, stopping
// rule, x0 = 0 and fixed-order reductions) for bulk and correction sources,
// and each right-hand side's arithmetic does not depend on its batch mates,
// so the correction term is an unbiased estimate of the LP bias.
#include <math.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace tsm {

namespace {

// out = bulk / N_LP + (hp - lpc) / N_HP; *bad is set when a value is not finite
__global__ void combine_kernel(const double* __restrict__ bulk, const double* __restrict__ hp,
                               const double* __restrict__ lpc, double inv_lp, double inv_hp, size_t n,
                               double* __restrict__ out, int* __restrict__ bad) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double e = bulk[i] * inv_lp;
  if (inv_hp != 0.0) e += (hp[i] - lpc[i]) * inv_hp;
  out[i] = e;
  if (!isfinite(e)) *bad = 1;
}

struct Accum {
  int iters_total = 0, iters_max = 0, not_conv = 0;
  double res_max = 0.0;
  void add(const std::vector<tsm_solve_stats>& st, int n) {
    for (int k = 0; k < n; ++k) {
      iters_total += st[k].iterations;
      iters_max = std::max(iters_max, st[k].iterations);
      res_max = std::max(res_max, st[k].true_residual);
      not_conv += !st[k].converged;
    }
  }
  void merge(const Accum& o) {
    iters_total += o.iters_total;
    iters_max = std::max(iters_max, o.iters_max);
    res_max = std::max(res_max, o.res_max);
    not_conv += o.not_conv;
  }
};

// The correction solves run on a second stream, beside the bulk, unless
// TSM_STREAMS=1 (measurements) or the per-kernel profiler is on.
bool concurrent_correction() {
  static const bool on = [] {
    const char* e = getenv("TSM_STREAMS");
    return !(e && atoi(e) == 1);
  }();
  return on && !profiling();
}

// Solve sources [first, first + n) with `solver` and add their loops to acc.
int solve_and_contract(tsm_gauge* g, const tsm_params* p, int solver, double rho, uint64_t first, int n,
                       int batch, DevBuf& sol, double* acc, Accum& a, cudaStream_t s, int slot) {
  // loops are contracted in FP64 for the all-FP64 solver and in FP32 otherwise
  const int op = (solver_kind(solver) == TSM_SOLVER_F64) ? TSM_F64 : TSM_F32;
  std::vector<tsm_solve_stats> st(batch);
  for (int k0 = 0; k0 < n; k0 += batch) {
    const int nb = std::min(batch, n - k0);
    TSM_TRY(sol.reserve(tsm_spinor_bytes(g, op, nb)));
    int rc = solve_batch_impl(g, p->kappa, p->mu, solver, rho, p->max_iter, nb, nullptr, 0, p->noise_seed,
                              first + k0, op, sol.p, 0, st.data(), s, slot);
    if (rc != TSM_OK && rc != TSM_ERR_NOT_CONVERGED) return rc;
    a.add(st, nb);
    TSM_TRY(contract_loops(g, p->kappa, p->mu, op, sol.p, nb, p->n_mom, p->mom, acc, 1, s, slot));
  }
  return TSM_OK;
}

// Batch sizes solve_and_contract uses for n sources in batches of `batch`.
std::vector<int> batch_sizes(int n, int batch) {
  std::vector<int> v;
  if (n <= 0) return v;
  v.push_back(std::min(batch, n));
  if (n > batch && n % batch) v.push_back(n % batch);
  return v;
}

// Everything the two concurrent halves of a TSM need -- solver and
// contraction workspaces, the insertion table, the autotuned launch shapes,
// the solvers' iteration-chunk graphs, the solution buffers -- is allocated,
// tuned and captured here, on the calling thread, before the worker thread
// starts.  During the concurrent phase the two threads then only enqueue
// work and replay graphs: no device allocation, free, autotuner timing run
// or stream capture happens on one thread while the other enqueues.
int prepare_tsm(tsm_gauge* g, const tsm_params* p, int batch, cudaStream_t s) {
  const int lp_op = (solver_kind(p->lp_solver) == TSM_SOLVER_F64) ? TSM_F64 : TSM_F32;
  const int hp_op = (solver_kind(p->hp_solver) == TSM_SOLVER_F64) ? TSM_F64 : TSM_F32;
  for (int nb : batch_sizes(p->n_lp, batch)) {
    TSM_TRY(prepare_solve(g, p->lp_solver, nb, p->kappa, p->mu, 0, s));
    TSM_TRY(prepare_contract(g, lp_op, nb, p->n_mom, p->mom, 0, s));
  }
  size_t sol2 = 0;
  for (int nb : batch_sizes(p->n_hp, batch)) {
    TSM_TRY(prepare_solve(g, p->hp_solver, nb, p->kappa, p->mu, 1, s));
    TSM_TRY(prepare_solve(g, p->lp_solver, nb, p->kappa, p->mu, 1, s));
    TSM_TRY(prepare_contract(g, hp_op, nb, p->n_mom, p->mom, 1, s));
    TSM_TRY(prepare_contract(g, lp_op, nb, p->n_mom, p->mom, 1, s));
    sol2 = std::max(sol2, std::max(tsm_spinor_bytes(g, hp_op, nb), tsm_spinor_bytes(g, lp_op, nb)));
  }
  TSM_TRY(g->tsm_sol.reserve(tsm_spinor_bytes(g, lp_op, std::min(batch, p->n_lp))));
  if (sol2) TSM_TRY(g->tsm_sol2.reserve(sol2));
  TSM_CUDA(cudaStreamSynchronize(s));
  return TSM_OK;
}

}  // namespace

}  // namespace tsm

using namespace tsm;

namespace tsm {

// Shared body: the estimate is left in est_dev (device) and, when the host
// pointers are given, copied out.
static int run_tsm(tsm_gauge* g, const tsm_params* p, double* est_dev, double* parts_dev, double* loops_host,
                   double* parts_host, tsm_stats* stats, void* stream) {
  if (!g || !p) return fail(TSM_ERR_INVALID_ARG, "tsm_solve_tsm: NULL argument");
  if (p->n_lp < 1 || p->n_hp < 0) return fail(TSM_ERR_INVALID_ARG, "need n_lp >= 1 and n_hp >= 0");
  if (p->n_mom < 1 || !p->mom) return fail(TSM_ERR_INVALID_ARG, "need at least one momentum");
  for (int solver : {p->lp_solver, p->hp_solver}) {
    if (solver_kind(solver) < 0) return fail(TSM_ERR_INVALID_ARG, "bad solver");
    if ((solver & TSM_SOLVER_EO) && !eo_lattice(g->geom))
      return fail(TSM_ERR_INVALID_ARG, "even-odd needs even extents in all four directions");
    const unsigned need = solver_link_precs(solver);
    if ((g->precisions & need) != need)
      return fail(TSM_ERR_INVALID_ARG, "solver %d needs gauge copies 0x%x", solver, need);
  }
  if (!(p->rho_lp > 0 && p->rho_lp < 1) || !(p->rho_hp > 0 && p->rho_hp < 1))
    return fail(TSM_ERR_INVALID_ARG, "rho_lp and rho_hp must lie in (0, 1)");
  if (p->max_iter < 1 || !(p->kappa > 0) || !isfinite(p->mu)) return fail(TSM_ERR_INVALID_ARG, "bad max_iter/kappa/mu");
  TSM_CUDA(cudaSetDevice(g->ctx->device));
  cudaStream_t s = pick_stream(g, stream);
  const auto t0 = std::chrono::steady_clock::now();
  const int batch = p->nrhs_per_launch > 0 ? std::min(p->nrhs_per_launch, 1024) : 12;
  const size_t n_out = (size_t)160 * p->n_mom * g->geom.L[3] * 2;
  std::lock_guard<std::mutex> lock(g->tsm_mu);
  TSM_TRY(g->tsm_acc.reserve(sizeof(double) * n_out * 4 + 16));
  double* bulk = g->tsm_acc.as<double>();
  double* hp = bulk + n_out;
  double* lpc = hp + n_out;
  double* est = est_dev ? est_dev : lpc + n_out;
  int* bad = reinterpret_cast<int*>(lpc + 2 * n_out);  // non-finite flag of the estimate
  TSM_CUDA(cudaMemsetAsync(bulk, 0, sizeof(double) * n_out * 3, s));
  TSM_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  Accum lp_a, hp_a, lpc_a;
  const uint64_t c0 = (uint64_t)p->n_lp;
  if (p->n_hp == 0 || !concurrent_correction()) {
    TSM_TRY(solve_and_contract(g, p, p->lp_solver, p->rho_lp, 0, p->n_lp, batch, g->tsm_sol, bulk, lp_a, s, 0));
    if (p->n_hp > 0) {
      TSM_TRY(solve_and_contract(g, p, p->hp_solver, p->rho_hp, c0, p->n_hp, batch, g->tsm_sol, hp, hp_a, s, 0));
      TSM_TRY(solve_and_contract(g, p, p->lp_solver, p->rho_lp, c0, p->n_hp, batch, g->tsm_sol, lpc, lpc_a, s, 0));
    }
  } else {
    // The correction sources' HP and LP solves (small batches whose kernels
    // leave HBM and SMs partly idle) run on a second stream from a worker
    // thread, beside the bulk LP solves on the caller's stream.  Each side
    // has its own workspaces (slot 1) and solution buffer; the host waits of
    // the solvers' convergence checks happen in each thread independently.
    if (!g->aux_stream) {
      // The correction chain (many small latency-bound launches) gets the
      // highest stream priority, so that its blocks are scheduled beside the
      // bulk's arithmetic-bound blocks as soon as slots free up.
      // TSM_AUX_PRIORITY=0 creates it at the default priority (measurements).
      static const bool prio = [] {
        const char* e = getenv("TSM_AUX_PRIORITY");
        return !(e && atoi(e) == 0);
      }();
      int least = 0, greatest = 0;
      TSM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
      TSM_CUDA(cudaStreamCreateWithPriority(&g->aux_stream, cudaStreamNonBlocking, prio ? greatest : least));
      TSM_CUDA(cudaEventCreateWithFlags(&g->aux_ev[0], cudaEventDisableTiming));
      TSM_CUDA(cudaEventCreateWithFlags(&g->aux_ev[1], cudaEventDisableTiming));
    }
    TSM_TRY(prepare_tsm(g, p, batch, s));
    cudaStream_t s2 = g->aux_stream;
    TSM_CUDA(cudaEventRecord(g->aux_ev[0], s));  // accumulators cleared
    TSM_CUDA(cudaStreamWaitEvent(s2, g->aux_ev[0], 0));
    int rc2 = TSM_OK;
    std::string err2;
    std::thread worker([&] {
      const cudaError_t e = cudaSetDevice(g->ctx->device);
      if (e != cudaSuccess) {
        rc2 = cuda_status(e, "cudaSetDevice", __FILE__, __LINE__);
      } else {
        rc2 = solve_and_contract(g, p, p->hp_solver, p->rho_hp, c0, p->n_hp, batch, g->tsm_sol2, hp, hp_a, s2, 1);
        if (rc2 == TSM_OK)
          rc2 = solve_and_contract(g, p, p->lp_solver, p->rho_lp, c0, p->n_hp, batch, g->tsm_sol2, lpc, lpc_a, s2, 1);
      }
      if (rc2 != TSM_OK) err2 = tsm_last_error();  // the message is thread-local
    });
    const int rc1 = solve_and_contract(g, p, p->lp_solver, p->rho_lp, 0, p->n_lp, batch, g->tsm_sol, bulk, lp_a, s, 0);
    worker.join();
    TSM_CUDA(cudaEventRecord(g->aux_ev[1], s2));  // the caller's stream continues after both
    TSM_CUDA(cudaStreamWaitEvent(s, g->aux_ev[1], 0));
    if (rc1 != TSM_OK) return rc1;
    if (rc2 != TSM_OK) return fail(rc2, "%s", err2.c_str());
  }
  lp_a.merge(lpc_a);
  const int bs = 256;
  count_launches(1);
  combine_kernel<<<(unsigned)((n_out + bs - 1) / bs), bs, 0, s>>>(bulk, hp, lpc, 1.0 / p->n_lp,
                                                                  p->n_hp ? 1.0 / p->n_hp : 0.0, n_out, est, bad);
  TSM_CUDA(cudaGetLastError());
  if (parts_dev) TSM_CUDA(cudaMemcpyAsync(parts_dev, bulk, sizeof(double) * n_out * 3, cudaMemcpyDeviceToDevice, s));
  if (loops_host) TSM_CUDA(cudaMemcpyAsync(loops_host, est, sizeof(double) * n_out, cudaMemcpyDeviceToHost, s));
  if (parts_host) TSM_CUDA(cudaMemcpyAsync(parts_host, bulk, sizeof(double) * n_out * 3, cudaMemcpyDeviceToHost, s));
  int bad_host = 0;
  if (loops_host) TSM_CUDA(cudaMemcpyAsync(&bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (loops_host || parts_host || stats) TSM_CUDA(cudaStreamSynchronize(s));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->lp_iterations_total = lp_a.iters_total;
    stats->lp_max_iterations = lp_a.iters_max;
    stats->lp_max_true_residual = lp_a.res_max;
    stats->hp_iterations_total = hp_a.iters_total;
    stats->hp_max_iterations = hp_a.iters_max;
    stats->hp_max_true_residual = hp_a.res_max;
    stats->n_not_converged = lp_a.not_conv + hp_a.not_conv;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (loops_host && bad_host) return fail(TSM_ERR_NONFINITE, "non-finite loop value");
  if (lp_a.not_conv + hp_a.not_conv)
    return fail(TSM_ERR_NOT_CONVERGED, "%d solves missed rho", lp_a.not_conv + hp_a.not_conv);
  return TSM_OK;
}

}  // namespace tsm

extern "C" int tsm_solve_tsm(tsm_gauge* g, const tsm_params* p, double* loops_host, double* parts_host,
                             tsm_stats* stats, void* stream) {
  if (!loops_host) return fail(TSM_ERR_INVALID_ARG, "tsm_solve_tsm: loops_host is NULL");
  return run_tsm(g, p, nullptr, nullptr, loops_host, parts_host, stats, stream);
}

extern "C" int tsm_solve_tsm_dev(tsm_gauge* g, const tsm_params* p, double* loops_dev, double* parts_dev,
                                 tsm_stats* stats, void* stream) {
  if (!loops_dev) return fail(TSM_ERR_INVALID_ARG, "tsm_solve_tsm_dev: loops_dev is NULL");
  return run_tsm(g, p, loops_dev, parts_dev, nullptr, nullptr, stats, stream);
}
