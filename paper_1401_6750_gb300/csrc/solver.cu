// Conjugate gradient on M^dag M for Eq. 1 (M s = eta), batched over
// right-hand sides, in four precision configurations (Sec. 2.1: low-precision
// solves for the bulk of the TSM, high-precision corrections):
//
//   F64          sloppy = precise = FP64
//   F32_RELIABLE sloppy FP32 (links r12, vectors), FP64 true residual and FP64
//                solution accumulator (reliable updates, delta = 0.1)
//   LP_F16/BF16  sloppy 16-bit links (r12) and p, Ap (with a per-rhs scale),
//                FP32 x and r; FP32 precise operator for residual replacement
//
// Iteration k (per right-hand side, all in one batch):
//   K_mp   q = M p            |q|^2 -> alpha = |r|^2 / (sigma^2 |q|^2)
//   K_mdag Ap = M^dag q;  r -= alpha Ap;  x += alpha p;   |r|^2 -> beta, stop test
//   K_p    p = r + beta p    (stored as p / sigma_new)
// Scalars live on the device (RhsState) and are finalised by the last block
// of each reducing kernel, so a chunk of iterations is a fixed launch
// sequence, captured once as a CUDA graph and replayed until every right-hand
// side has stopped.  Global sums are FP64, reduced in a fixed order.
//
// Stopping rule: iterated |r| <= rho |b| (b = M^dag eta), then the true
// residual b - M^dag M x with the precise operator decides; otherwise the
// iteration restarts from the true residual (p = r), up to max_iter.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "dslash.cuh"
#include "internal.h"
#include "solver_kernels.cuh"

namespace tsm {

namespace {

using namespace solverk;

}  // namespace

// ---------------------------------------------------------------- workspace
struct SolverWorkspace {
  std::mutex mu;  // held for a whole solve
  UseOrder order;  // orders the GPU use across the callers' streams
  int kind = -1;
  int cap = 0;  // right-hand sides allocated
  int nblk = 0;
  DevBuf st, partial, counter, mask, b, x, r, p, q, t, xacc;
  RhsState* h_st = nullptr;
  int* h_mask = nullptr;
  std::map<int, cudaGraphExec_t> graphs;  // chunk graphs per nrhs
  int nr_s = 1, nr_p = 1;                  // autotuned rhs per thread (sloppy, precise operator)
  double graph_kappa = 0.0, graph_mup = 0.0;
  ~SolverWorkspace() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    if (h_st) cudaFreeHost(h_st);
    if (h_mask) cudaFreeHost(h_mask);
  }
};

void SolverWsDeleter::operator()(SolverWorkspace* w) const { delete w; }

int solver_precise_prec(int solver) {
  solver &= ~TSM_SOLVER_EO;
  return (solver == TSM_SOLVER_F64 || solver == TSM_SOLVER_F32_RELIABLE) ? TSM_F64 : TSM_F32;
}
int solver_output_prec(int solver) {
  solver &= ~TSM_SOLVER_EO;
  return (solver == TSM_SOLVER_F64 || solver == TSM_SOLVER_F32_RELIABLE) ? TSM_F64 : TSM_F32;
}
unsigned solver_link_precs(int solver) {
  switch (solver & ~TSM_SOLVER_EO) {
    case TSM_SOLVER_F64: return TSM_PREC_BIT(TSM_F64);
    case TSM_SOLVER_F32_RELIABLE: return TSM_PREC_BIT(TSM_F32) | TSM_PREC_BIT(TSM_F64);
    case TSM_SOLVER_LP_F16: return TSM_PREC_BIT(TSM_F16) | TSM_PREC_BIT(TSM_F32);
    case TSM_SOLVER_LP_BF16: return TSM_PREC_BIT(TSM_BF16) | TSM_PREC_BIT(TSM_F32);
  }
  return 0;
}

namespace {

int chunk_iterations() {
  static int k = [] {
    const char* e = getenv("TSM_CG_CHUNK");
    int v = e ? atoi(e) : 8;
    return v > 0 ? v : 8;
  }();
  return k;
}
bool graphs_enabled() {
  static bool on = [] {
    const char* e = getenv("TSM_CUDA_GRAPHS");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <int KIND>
struct Solver {
  using T = Traits<KIND>;
  using Rs = typename T::Rs;
  using Rp = typename T::Rp;

  static int reserve(tsm_gauge* g, SolverWorkspace& w, int nrhs, cudaStream_t s) {
    if (w.cap >= nrhs) return TSM_OK;
    for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
    w.graphs.clear();
    const int V = g->geom.V;
    w.nblk = (V + DSLASH_BS - 1) / DSLASH_BS;
    TSM_TRY(w.st.reserve(sizeof(RhsState) * nrhs));
    TSM_TRY(w.partial.reserve(sizeof(double) * (size_t)nrhs * w.nblk));
    TSM_TRY(w.counter.reserve(sizeof(unsigned) * nrhs));
    // stream-ordered: a legacy-stream memset would implicitly synchronise with
    // (and so invalidate) a graph capture running on a blocking stream of
    // another host thread
    TSM_CUDA(cudaMemsetAsync(w.counter.p, 0, sizeof(unsigned) * nrhs, s));
    TSM_TRY(w.mask.reserve(sizeof(int) * nrhs));
    TSM_TRY(w.b.reserve(field_bytes(T::PP, V, nrhs)));
    TSM_TRY(w.t.reserve(field_bytes(T::PP, V, nrhs)));
    TSM_TRY(w.x.reserve(field_bytes(T::PA, V, nrhs)));
    TSM_TRY(w.r.reserve(field_bytes(T::PA, V, nrhs)));
    TSM_TRY(w.p.reserve(field_bytes(T::PS, V, nrhs)));
    TSM_TRY(w.q.reserve(field_bytes(T::PS, V, nrhs)));
    if (T::XACC) TSM_TRY(w.xacc.reserve(field_bytes(T::PXA, V, nrhs)));
    if (w.h_st) cudaFreeHost(w.h_st);
    if (w.h_mask) cudaFreeHost(w.h_mask);
    w.h_st = nullptr;
    w.h_mask = nullptr;
    TSM_CUDA(cudaMallocHost(&w.h_st, sizeof(RhsState) * nrhs));
    TSM_CUDA(cudaMallocHost(&w.h_mask, sizeof(int) * nrhs));
    w.cap = nrhs;
    return TSM_OK;
  }

  static DslashArgs args(const tsm_gauge* g, int pl, const void* in, double kappa, double tw, int nrhs) {
    DslashArgs a;
    a.g = g->geom;
    a.links = g->links[pl].p;
    a.in = in;
    a.nrhs = nrhs;
    a.nblk = (g->geom.V + DSLASH_BS - 1) / DSLASH_BS;
    set_coeffs(a, kappa, tw);
    return a;
  }

  static RedSlots slots(SolverWorkspace& w) { return RedSlots{w.partial.as<double>(), w.counter.as<unsigned>()}; }

  static double delta() {
    // TSM_RU_DELTA_<kind> overrides the residual-replacement threshold (measurement only)
    static const double d = [] {
      char name[32];
      snprintf(name, sizeof(name), "TSM_RU_DELTA_%d", KIND);
      const char* e = getenv(name);
      return e ? atof(e) : T::DELTA;
    }();
    return d;
  }

  static SolveParams params(const tsm_gauge* g, double rho, int max_iter) {
    SolveParams p;
    const double rc = cert_rho(rho, T::CERT);
    p.rho2 = rc * rc;
    p.delta2 = delta() * delta();
    p.inv_ncomp = 1.0 / (12.0 * (double)g->geom.V);
    p.max_iter = max_iter;
    p.scaled = T::SCALED ? 1 : 0;
    return p;
  }

  // One CG iteration for all active right-hand sides.
  static void iteration(const tsm_gauge* g, SolverWorkspace& w, int nrhs, double kappa, double mup,
                        const SolveParams& prm, cudaStream_t s) {
    count_launches(3);
    const size_t V = (size_t)g->geom.V;
    {
      EpiMp<Rs, T::PS> e{w.q.p, V, w.st.as<RhsState>(), slots(w)};
      launch_dslash<Rs, -1, T::PS, T::PLs>(w.nr_s, args(g, T::PLs, w.p.p, kappa, mup, nrhs), e, s);
    }
    {
      EpiCG<Rs, T::PA, T::PS> e{w.r.p, w.x.p, w.p.p, V, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash<Rs, +1, T::PS, T::PLs>(w.nr_s, args(g, T::PLs, w.q.p, kappa, -mup, nrhs), e, s);
    }
    dim3 eg((g->geom.V + EW_BS - 1) / EW_BS, nrhs);
    k_pupdate<T::PA, T::PS><<<eg, EW_BS, 0, s>>>(w.r.p, w.p.p, w.st.as<RhsState>(), 0, g->geom.V);
  }

  static const char* pname() {
    return T::PS == TSM_F64 ? "f64" : (T::PS == TSM_F32 ? "f32" : (T::PS == TSM_F16 ? "f16" : "bf16"));
  }

  // One iteration with each kernel bracketed by CUDA events (profiling mode).
  static int iteration_profiled(const tsm_gauge* g, SolverWorkspace& w, int nrhs, double kappa, double mup,
                                const SolveParams& prm, cudaStream_t s, int n_active) {
    count_launches(3);
    const size_t V = (size_t)g->geom.V;
    EventPair e1, e2, e3;
    TSM_TRY(e1.begin(s));
    {
      EpiMp<Rs, T::PS> e{w.q.p, V, w.st.as<RhsState>(), slots(w)};
      launch_dslash<Rs, -1, T::PS, T::PLs>(w.nr_s, args(g, T::PLs, w.p.p, kappa, mup, nrhs), e, s);
    }
    TSM_TRY(e1.end(s));
    TSM_TRY(e2.begin(s));
    {
      EpiCG<Rs, T::PA, T::PS> e{w.r.p, w.x.p, w.p.p, V, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash<Rs, +1, T::PS, T::PLs>(w.nr_s, args(g, T::PLs, w.q.p, kappa, -mup, nrhs), e, s);
    }
    TSM_TRY(e2.end(s));
    TSM_TRY(e3.begin(s));
    dim3 eg((g->geom.V + EW_BS - 1) / EW_BS, nrhs);
    k_pupdate<T::PA, T::PS><<<eg, EW_BS, 0, s>>>(w.r.p, w.p.p, w.st.as<RhsState>(), 0, g->geom.V);
    TSM_TRY(e3.end(s));
    TSM_CUDA(cudaGetLastError());
    const double v = (double)V, n = (double)n_active;
    const double ls = link_site_bytes(T::PLs), bs = spinor_site_bytes(T::PS), ba = spinor_site_bytes(T::PA);
    char name[48];
    snprintf(name, sizeof(name), "cg_Mp_%s", pname());
    prof_add(name, e1.seconds(), v * (ls + n * 2 * bs), v * n * (1392.0 + 48.0));
    snprintf(name, sizeof(name), "cg_MdagQ_update_%s", pname());
    prof_add(name, e2.seconds(), v * (ls + n * (2 * bs + 4 * ba)), v * n * (1392.0 + 96.0 + 48.0));
    snprintf(name, sizeof(name), "cg_p_update_%s", pname());
    prof_add(name, e3.seconds(), v * n * (ba + 2 * bs), v * n * 72.0);
    return TSM_OK;
  }

  static int run_chunk(const tsm_gauge* g, SolverWorkspace& w, int nrhs, double kappa, double mup,
                       const SolveParams& prm, cudaStream_t s) {
    const int k = chunk_iterations();
    if (!graphs_enabled()) {
      for (int it = 0; it < k; ++it) iteration(g, w, nrhs, kappa, mup, prm, s);
      TSM_CUDA(cudaGetLastError());
      return TSM_OK;
    }
    cudaGraphExec_t exec;  // kernel arguments carry kappa and mu': a change invalidates the cached graphs
    TSM_TRY(ensure_graph(g, w, nrhs, kappa, mup, prm, s, &exec));
    TSM_CUDA(cudaGraphLaunch(exec, s));
    count_launches(3LL * k);
    return TSM_OK;
  }

  // The chunk graph for nrhs, captured on s if not cached (kernel arguments
  // hold workspace pointers, kappa, mu' and solver constants only; what a
  // solve changes lives in the device state).
  static int ensure_graph(const tsm_gauge* g, SolverWorkspace& w, int nrhs, double kappa, double mup,
                          const SolveParams& prm, cudaStream_t s, cudaGraphExec_t* out) {
    if (w.graph_kappa != kappa || w.graph_mup != mup) {
      for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
      w.graphs.clear();
      w.graph_kappa = kappa;
      w.graph_mup = mup;
    }
    auto found = w.graphs.find(nrhs);
    if (found == w.graphs.end()) {
      const int k = chunk_iterations();
      cudaGraph_t graph;
      TSM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      for (int i = 0; i < k; ++i) iteration(g, w, nrhs, kappa, mup, prm, s);
      count_launches(-3LL * k);  // captured, not launched
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      cudaGraphExec_t exec;
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      found = w.graphs.emplace(nrhs, exec).first;
    }
    *out = found->second;
    return TSM_OK;
  }

  // right-hand sides per thread of both operators (autotuned); a change drops the cached graphs
  static int set_shapes(tsm_gauge* g, SolverWorkspace& w, int nrhs, cudaStream_t s) {
    int nr_s = 1, nr_p = 1;
    TSM_TRY(tuned_nr(g, T::PS, T::PLs, nrhs, s, &nr_s));
    TSM_TRY(tuned_nr(g, T::PP, T::PLp, nrhs, s, &nr_p));
    if (nr_s != w.nr_s) {  // captured graphs bake in the launch shape
      for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
      w.graphs.clear();
    }
    w.nr_s = nr_s;
    w.nr_p = nr_p;
    return TSM_OK;
  }

  // residual replacement for the rhs in w.mask: r = b - M^dag M x_true
  static int replace_residual(const tsm_gauge* g, SolverWorkspace& w, int nrhs, double kappa, double mup,
                              const SolveParams& prm, cudaStream_t s) {
    const size_t V = (size_t)g->geom.V;
    dim3 eg((g->geom.V + EW_BS - 1) / EW_BS, nrhs);
    const void* xsrc = w.x.p;
    count_launches(T::XACC ? 4 : 3);
    if (T::XACC) {
      k_fold<T::PA, T::PXA><<<eg, EW_BS, 0, s>>>(w.x.p, w.xacc.p, w.mask.as<int>(), g->geom.V);
      xsrc = w.xacc.p;
    }
    {
      EpiStoreMasked<Rp, T::PP> e{w.t.p, V, w.mask.as<int>(), RedSlots{nullptr, nullptr}};
      launch_dslash<Rp, -1, T::PX, T::PLp>(w.nr_p, args(g, T::PLp, xsrc, kappa, mup, nrhs), e, s);
    }
    {
      EpiResidual<Rp, T::PP, T::PA> e{w.b.p, w.r.p, V, w.mask.as<int>(), w.st.as<RhsState>(), slots(w), prm};
      launch_dslash<Rp, +1, T::PP, T::PLp>(w.nr_p, args(g, T::PLp, w.t.p, kappa, -mup, nrhs), e, s);
    }
    k_pupdate<T::PA, T::PS><<<eg, EW_BS, 0, s>>>(w.r.p, w.p.p, w.st.as<RhsState>(), 1, g->geom.V);
    TSM_CUDA(cudaGetLastError());
    return TSM_OK;
  }

  // Solve for eta already in w.t (precise precision).
  static int solve(tsm_gauge* g, SolverWorkspace& w, int nrhs, double kappa, double mu, double rho, int max_iter,
                   int out_prec, void* x_out, int gamma5_out, tsm_solve_stats* stats, cudaStream_t s) {
    const double mup = 2.0 * kappa * mu;
    const SolveParams prm = params(g, rho, max_iter);
    const size_t V = (size_t)g->geom.V;
    TSM_TRY(set_shapes(g, w, nrhs, s));
    dim3 eg((g->geom.V + EW_BS - 1) / EW_BS, nrhs);
    // b = M^dag eta (precise), state initialisation
    count_launches(2);
    {
      EpiInitB<Rp, T::PP> e{w.b.p, V, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash<Rp, +1, T::PP, T::PLp>(w.nr_p, args(g, T::PLp, w.t.p, kappa, -mup, nrhs), e, s);
    }
    k_init<T::PP, T::PA, T::PS, T::XACC, T::PXA>
        <<<eg, EW_BS, 0, s>>>(w.b.p, w.r.p, w.x.p, w.p.p, w.xacc.p, w.st.as<RhsState>(), g->geom.V);
    TSM_CUDA(cudaGetLastError());
    const int k = chunk_iterations();
    const long long limit = (long long)max_iter / k + 64;  // host-side bound on chunks
    for (long long round = 0;; ++round) {
      TSM_CUDA(cudaMemcpyAsync(w.h_st, w.st.p, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost, s));
      TSM_CUDA(cudaStreamSynchronize(s));
      bool any_ru = false, any_active = false;
      for (int r = 0; r < nrhs; ++r) {
        const RhsState& h = w.h_st[r];
        const int m = (h.active && h.need_ru) || h.status == ST_ITER_CONV || h.status == ST_MAXITER;
        w.h_mask[r] = m;
        any_ru |= (m != 0);
      }
      if (any_ru) {
        TSM_CUDA(cudaMemcpyAsync(w.mask.p, w.h_mask, sizeof(int) * nrhs, cudaMemcpyHostToDevice, s));
        TSM_TRY(replace_residual(g, w, nrhs, kappa, mup, prm, s));
        TSM_CUDA(cudaMemcpyAsync(w.h_st, w.st.p, sizeof(RhsState) * nrhs, cudaMemcpyDeviceToHost, s));
        TSM_CUDA(cudaStreamSynchronize(s));
      }
      for (int r = 0; r < nrhs; ++r) any_active |= (w.h_st[r].active != 0);
      if (!any_active) break;
      if (round > limit * chunk_iterations()) return fail(TSM_ERR_CUDA, "solver exceeded its chunk bound");
      if (profiling()) {
        int n_active = 0;
        for (int r = 0; r < nrhs; ++r) n_active += (w.h_st[r].active != 0);
        TSM_TRY(iteration_profiled(g, w, nrhs, kappa, mup, prm, s, n_active));
      } else {
        TSM_TRY(run_chunk(g, w, nrhs, kappa, mup, prm, s));
      }
    }
    count_launches(1);
    // solution (x_acc + x for the reliable-update solver) in the precise precision, into w.t
    k_output<T::PA, T::PP, T::XACC, T::PXA><<<eg, EW_BS, 0, s>>>(w.x.p, w.xacc.p, w.t.p, gamma5_out,
                                                          g->geom.V);
    TSM_TRY(spinor_convert(g, out_prec, x_out, T::PP, w.t.p, nrhs, 0, s));
    int bad = 0;
    for (int r = 0; r < nrhs; ++r) {
      const RhsState& h = w.h_st[r];
      const int ok = (h.status == ST_DONE);
      bad += !ok;
      if (stats) {
        stats[r].iterations = h.iter;
        stats[r].reliable_updates = h.n_ru;
        stats[r].converged = ok;
        stats[r].restarts = h.restarts;
        stats[r].true_residual = h.bb > 0 ? sqrt(h.true_rr / h.bb) : 0.0;
      }
    }
    for (int r = 0; r < nrhs; ++r)
      if (w.h_st[r].status == ST_BREAKDOWN) return fail(TSM_ERR_NONFINITE, "solver breakdown (non-finite residual)");
    if (bad) return fail(TSM_ERR_NOT_CONVERGED, "%d of %d right-hand sides missed rho", bad, nrhs);
    return TSM_OK;
  }
};

template <int KIND>
int solve_kind(tsm_gauge* g, double kappa, double mu, double rho, int max_iter, int nrhs, const void* eta,
               int eta_prec, uint64_t seed, uint64_t first, int out_prec, void* x_out, int gamma5_io,
               tsm_solve_stats* stats, cudaStream_t s, int slot) {
  using T = Traits<KIND>;
  SolverWorkspace* wp;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    auto& ws = g->solver_ws[KIND + 64 * slot];
    if (!ws) ws.reset(new SolverWorkspace());
    wp = ws.get();
  }
  SolverWorkspace& w = *wp;
  std::lock_guard<std::mutex> wlock(w.mu);
  w.kind = KIND;
  TSM_TRY(w.order.enter(s));
  TSM_TRY(Solver<KIND>::reserve(g, w, nrhs, s));
  if (eta) {
    TSM_TRY(spinor_convert(g, T::PP, w.t.p, eta_prec, eta, nrhs, gamma5_io, s));
  } else {
    TSM_TRY(make_sources(g, seed, first, nrhs, T::PP, w.t.p, s));
  }
  const int rc = Solver<KIND>::solve(g, w, nrhs, kappa, mu, rho, max_iter, out_prec, x_out, gamma5_io, stats, s);
  const int rc_order = w.order.leave(s);
  return rc != TSM_OK ? rc : rc_order;
}

// Workspace and tuned launch shapes of a solve of nrhs right-hand sides on
// `slot`, made ahead of the solve (which then allocates and times nothing).
template <int KIND>
int prepare_kind(tsm_gauge* g, int nrhs, double kappa, double mu, int slot, cudaStream_t s) {
  SolverWorkspace* wp;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    auto& ws = g->solver_ws[KIND + 64 * slot];
    if (!ws) ws.reset(new SolverWorkspace());
    wp = ws.get();
  }
  SolverWorkspace& w = *wp;
  std::lock_guard<std::mutex> wlock(w.mu);
  w.kind = KIND;
  TSM_TRY(w.order.enter(s));
  TSM_TRY(Solver<KIND>::reserve(g, w, nrhs, s));
  TSM_TRY(Solver<KIND>::set_shapes(g, w, nrhs, s));
  if (graphs_enabled() && !profiling()) {  // the chunk graph too: a solve then captures nothing
    cudaGraphExec_t exec;
    TSM_TRY(Solver<KIND>::ensure_graph(g, w, nrhs, kappa, 2.0 * kappa * mu, Solver<KIND>::params(g, 0.5, 1), s,
                                       &exec));
  }
  return w.order.leave(s);
}

}  // namespace

int prepare_solve(tsm_gauge* g, int solver, int nrhs, double kappa, double mu, int slot, cudaStream_t s) {
  if (slot < 0 || slot > 1 || nrhs < 1) return fail(TSM_ERR_INVALID_ARG, "prepare_solve: slot %d, nrhs %d", slot, nrhs);
  if (solver & TSM_SOLVER_EO) return prepare_eo(g, solver, nrhs, kappa, mu, slot, s);
  switch (solver) {
    case TSM_SOLVER_F64: return prepare_kind<TSM_SOLVER_F64>(g, nrhs, kappa, mu, slot, s);
    case TSM_SOLVER_F32_RELIABLE: return prepare_kind<TSM_SOLVER_F32_RELIABLE>(g, nrhs, kappa, mu, slot, s);
    case TSM_SOLVER_LP_F16: return prepare_kind<TSM_SOLVER_LP_F16>(g, nrhs, kappa, mu, slot, s);
    case TSM_SOLVER_LP_BF16: return prepare_kind<TSM_SOLVER_LP_BF16>(g, nrhs, kappa, mu, slot, s);
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown solver %d", solver);
}

// eta == nullptr: Z4 sources (seed, first) are generated in place.
int solve_batch_impl(tsm_gauge* g, double kappa, double mu, int solver, double rho, int max_iter, int nrhs,
                     const void* eta, int eta_prec, uint64_t seed, uint64_t first, int out_prec, void* x_out,
                     int gamma5_io, tsm_solve_stats* stats, cudaStream_t s, int slot) {
  if (slot < 0 || slot > 1) return fail(TSM_ERR_INVALID_ARG, "workspace slot %d", slot);
  const unsigned need = solver_link_precs(solver);
  if ((g->precisions & need) != need)
    return fail(TSM_ERR_INVALID_ARG, "solver %d needs gauge copies 0x%x, gauge has 0x%x", solver, need,
                g->precisions);
  if (solver & TSM_SOLVER_EO)
    return solve_batch_eo(g, kappa, mu, solver, rho, max_iter, nrhs, eta, eta_prec, seed, first, out_prec, x_out,
                          gamma5_io, stats, s, slot);
  switch (solver) {
    case TSM_SOLVER_F64:
      return solve_kind<TSM_SOLVER_F64>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first, out_prec,
                                        x_out, gamma5_io, stats, s, slot);
    case TSM_SOLVER_F32_RELIABLE:
      return solve_kind<TSM_SOLVER_F32_RELIABLE>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                                 out_prec, x_out, gamma5_io, stats, s, slot);
    case TSM_SOLVER_LP_F16:
      return solve_kind<TSM_SOLVER_LP_F16>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                           out_prec, x_out, gamma5_io, stats, s, slot);
    case TSM_SOLVER_LP_BF16:
      return solve_kind<TSM_SOLVER_LP_BF16>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                            out_prec, x_out, gamma5_io, stats, s, slot);
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown solver %d", solver);
}

}  // namespace tsm
