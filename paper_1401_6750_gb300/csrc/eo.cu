// Even-odd (Schur complement) preconditioned solves of Eq. 1 (every lattice
// extent even, so that every hop joins sites of opposite parity).
//
// With sites split by parity, M = [[M_ee, M_eo], [M_oe, M_oo]] where
// M_ee = M_oo = 1 + i mu' g5 is site-local and M_eo = -kappa H_eo is the
// hopping part.  M s = eta is solved through the odd-site system
//   Mhat s_o = eta_o - M_oe M_ee^{-1} eta_e,   Mhat = M_oo - M_oe M_ee^{-1} M_eo,
//   s_e = M_ee^{-1} (eta_e - M_eo s_o),        M_ee^{-1} = (1 - i mu' g5) / (1 + mu'^2),
// by CG on Mhat^dag Mhat (Mhat^dag = g5 Mhat(-mu) g5).  One application of
// Mhat is two half-volume hops:
//   A: t_e = M_ee^{-1} (-kappa H_eo v_o)
//   B: out_o = (1 + i mu' g5) v_o + kappa H_oe t_e
// so an iteration costs the stencil work of the unpreconditioned CG on
// vectors of half the size, and Mhat^dag Mhat is better conditioned.
// Solutions are returned on all sites; the stopping rule is that of the
// unpreconditioned solvers applied to the normal equations of Mhat.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

#include "dslash.cuh"
#include "internal.h"
#include "solver_kernels.cuh"
#include "tc_hop.cuh"

namespace tsm {

namespace {

using namespace solverk;

// full (V sites) -> even and odd halves (V/2 each), nrhs fields
template <int P>
__global__ void k_gather_eo(const void* full, void* even, void* odd, Geom g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= g.V) return;
  int c[4];
  site_coords(g, i, c);
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  cplx<ew_real<P>> v[12];
  SpinorIO<P>::load(full, (size_t)g.V, rhs, i, v);
  SpinorIO<P>::store(par ? odd : even, (size_t)g.V / 2, rhs, i >> 1, v);
}

// even and odd halves -> full, optionally times g5
template <int PO, int PI>
__global__ void k_scatter_eo(void* full, const void* even, const void* odd, Geom g, int gamma5) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= g.V) return;
  int c[4];
  site_coords(g, i, c);
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  using R = ew_real<PO, PI>;
  cplx<R> v[12];
  SpinorIO<PI>::load(par ? odd : even, (size_t)g.V / 2, rhs, i >> 1, v);
  if (gamma5) {
#pragma unroll
    for (int k = 6; k < 12; ++k) v[k] = mk<R>(-v[k].re, -v[k].im);
  }
  SpinorIO<PO>::store(full, (size_t)g.V, rhs, i, v);
}

// full -> even and odd halves, and diag_even = (cr + i ci g5) eta_e on the
// even sites, in one pass
template <int P>
__global__ void k_split_eo(const void* full, void* even, void* odd, void* diag_even, double cr, double ci, Geom g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= g.V) return;
  int c[4];
  site_coords(g, i, c);
  using R = ew_real<P>;
  cplx<R> v[12];
  SpinorIO<P>::load(full, (size_t)g.V, rhs, i, v);
  const size_t vh = (size_t)g.V / 2;
  if ((c[0] + c[1] + c[2] + c[3]) & 1) {
    SpinorIO<P>::store(odd, vh, rhs, i >> 1, v);
    return;
  }
  SpinorIO<P>::store(even, vh, rhs, i >> 1, v);
  const R a = (R)cr, b = (R)ci;
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = a * v[k] + (k < 6 ? b : -b) * times_i(v[k]);
  SpinorIO<P>::store(diag_even, vh, rhs, i >> 1, v);
}

}  // namespace

struct EoWorkspace {
  std::mutex mu;  // held for a whole solve
  UseOrder order;  // orders the GPU use across the callers' streams
  int cap = 0, nblk = 0;
  DevBuf st, partial, counter, mask, b, t1, tep, eta_e, x, r, p, q, tes, xacc, full;
  RhsState* h_st = nullptr;
  int* h_mask = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  double graph_kappa = 0.0, graph_mup = 0.0;
  int nr_s = 1, nr_p = 1;  // right-hand sides per thread (sloppy, precise operator)
  ~EoWorkspace() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    if (h_st) cudaFreeHost(h_st);
    if (h_mask) cudaFreeHost(h_mask);
  }
};
void EoWsDeleter::operator()(EoWorkspace* w) const { delete w; }

namespace {

// Right-hand sides per thread of the checkerboarded operator on fields of
// precision `prec`; TSM_EO_NR_<F64|F32|F16|BF16> override it (measurements).
int eo_nr(int prec) {
  if (prec == TSM_DS) return 1;  // float-float sums leave no registers for a second right-hand side
  static const int env[4] = {
      [] { const char* e = getenv("TSM_EO_NR_F64"); return e ? atoi(e) : 0; }(),
      [] { const char* e = getenv("TSM_EO_NR_F32"); return e ? atoi(e) : 0; }(),
      [] { const char* e = getenv("TSM_EO_NR_F16"); return e ? atoi(e) : 0; }(),
      [] { const char* e = getenv("TSM_EO_NR_BF16"); return e ? atoi(e) : 0; }(),
  };
  static const int dflt[4] = {1, 1, 1, 1};
  int nr = (prec >= 0 && prec < 4 && env[prec]) ? env[prec] : dflt[prec & 3];
  if (nr != 1 && nr != 2 && nr != 4) nr = 1;
  if (nr == 4 && prec == TSM_F64) nr = 2;
  return nr;
}

int eo_chunk() {
  static int k = [] {
    const char* e = getenv("TSM_CG_CHUNK");
    int v = e ? atoi(e) : 8;
    return v > 0 ? v : 8;
  }();
  return k;
}

template <int KIND>
struct SolverEO {
  using T = Traits<KIND>;
  using Rs = typename T::Rs;
  using Rp = typename T::Rp;

  static size_t half(int prec, int V, int n) { return (size_t)n * spinor_chunks(prec) * (size_t)(V / 2) * 16; }

  static int reserve(tsm_gauge* g, EoWorkspace& w, int nrhs, cudaStream_t s) {
    if (w.cap >= nrhs) return TSM_OK;
    for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
    w.graphs.clear();
    const int V = g->geom.V;
    w.nblk = (V / 2 + DSLASH_BS - 1) / DSLASH_BS;
    TSM_TRY(w.st.reserve(sizeof(RhsState) * nrhs));
    TSM_TRY(w.partial.reserve(sizeof(double) * (size_t)nrhs * w.nblk));
    TSM_TRY(w.counter.reserve(sizeof(unsigned) * nrhs));
    TSM_CUDA(cudaMemsetAsync(w.counter.p, 0, sizeof(unsigned) * nrhs, s));  // stream-ordered (see solver.cu)
    TSM_TRY(w.mask.reserve(sizeof(int) * nrhs));
    TSM_TRY(w.b.reserve(half(T::PP, V, nrhs)));
    TSM_TRY(w.t1.reserve(half(T::PP, V, nrhs)));
    TSM_TRY(w.tep.reserve(half(T::PP, V, nrhs)));
    TSM_TRY(w.eta_e.reserve(half(T::PP, V, nrhs)));
    TSM_TRY(w.x.reserve(half(T::PA, V, nrhs)));
    TSM_TRY(w.r.reserve(half(T::PA, V, nrhs)));
    TSM_TRY(w.p.reserve(half(T::PS, V, nrhs)));
    TSM_TRY(w.q.reserve(half(T::PS, V, nrhs)));
    TSM_TRY(w.tes.reserve(half(T::PS, V, nrhs)));
    if (T::XACC) TSM_TRY(w.xacc.reserve(half(T::PXA, V, nrhs)));
    TSM_TRY(w.full.reserve(2 * half(T::PP, V, nrhs)));
    if (w.h_st) cudaFreeHost(w.h_st);
    if (w.h_mask) cudaFreeHost(w.h_mask);
    w.h_st = nullptr;
    w.h_mask = nullptr;
    TSM_CUDA(cudaMallocHost(&w.h_st, sizeof(RhsState) * nrhs));
    TSM_CUDA(cudaMallocHost(&w.h_mask, sizeof(int) * nrhs));
    w.cap = nrhs;
    return TSM_OK;
  }

  static RedSlots slots(EoWorkspace& w) { return RedSlots{w.partial.as<double>(), w.counter.as<unsigned>()}; }

  // hop args: output parity `par`, input field `in`, center field `ctr` (may be null)
  static DslashArgs args(const tsm_gauge* g, int pl, const void* in, const void* ctr, int par, double kappa, double c0,
                         double c1, double h0, double h1, int nrhs) {
    DslashArgs a;
    a.g = g->geom;
    a.links = g->links[pl].p;
    a.in = in;
    a.nrhs = nrhs;
    a.nblk = (g->geom.V / 2 + DSLASH_BS - 1) / DSLASH_BS;
    set_coeffs(a, kappa, 0.0);
    set_eo(a, ctr, par, c0, c1, h0, h1);
    return a;
  }
  // step A (to even): t_e = M_ee(tau)^{-1} (-kappa H v_o); step B (to odd): (1 + i tau g5) v_o + kappa H t_e
  static DslashArgs step_a(const tsm_gauge* g, int pl, const void* in, double kappa, double tau, int nrhs) {
    const double d = 1.0 + tau * tau;
    return args(g, pl, in, nullptr, 0, kappa, 0.0, 0.0, -kappa / d, kappa * tau / d, nrhs);
  }
  static DslashArgs step_b(const tsm_gauge* g, int pl, const void* in, const void* ctr, double kappa, double tau,
                           int nrhs) {
    return args(g, pl, in, ctr, 1, kappa, 1.0, tau, kappa, 0.0, nrhs);
  }

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
    p.inv_ncomp = 1.0 / (12.0 * (double)(g->geom.V / 2));
    p.max_iter = max_iter;
    p.scaled = T::SCALED ? 1 : 0;
    return p;
  }

  static void iteration(const tsm_gauge* g, EoWorkspace& w, int nrhs, double kappa, double mup,
                        const SolveParams& prm, cudaStream_t s) {
    count_launches(5);
    const size_t Vh = (size_t)g->geom.V / 2;
    EpiStore<Rs, T::PS> es{w.tes.p, Vh, 0, RedSlots{nullptr, nullptr}};
    // q = Mhat p
    launch_dslash_eo_tc<Rs, -1, T::PS, T::PLs>(w.nr_s, step_a(g, T::PLs, w.p.p, kappa, mup, nrhs), es, s);
    {
      EpiMp<Rs, T::PS> e{w.q.p, Vh, w.st.as<RhsState>(), slots(w)};
      launch_dslash_eo_tc<Rs, -1, T::PS, T::PLs>(w.nr_s, step_b(g, T::PLs, w.tes.p, w.p.p, kappa, mup, nrhs), e, s);
    }
    // Ap = Mhat^dag q; r -= alpha Ap; x += alpha p
    launch_dslash_eo_tc<Rs, +1, T::PS, T::PLs>(w.nr_s, step_a(g, T::PLs, w.q.p, kappa, -mup, nrhs), es, s);
    {
      EpiCG<Rs, T::PA, T::PS> e{w.r.p, w.x.p, w.p.p, Vh, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash_eo_tc<Rs, +1, T::PS, T::PLs>(w.nr_s, step_b(g, T::PLs, w.tes.p, w.q.p, kappa, -mup, nrhs), e, s);
    }
    dim3 eg(((int)Vh + EW_BS - 1) / EW_BS, nrhs);
    k_pupdate<T::PA, T::PS><<<eg, EW_BS, 0, s>>>(w.r.p, w.p.p, w.st.as<RhsState>(), 0, (int)Vh);
  }

  static const char* pname() {
    return T::PS == TSM_F64 ? "f64" : (T::PS == TSM_F32 ? "f32" : (T::PS == TSM_F16 ? "f16" : "bf16"));
  }

  // One iteration with each launch timed on its own (profiling mode).  A
  // half-volume hop reads every link once and the input spinors of one
  // parity once; step B also reads the centre field.
  static int iteration_profiled(const tsm_gauge* g, EoWorkspace& w, int nrhs, double kappa, double mup,
                                const SolveParams& prm, cudaStream_t s, int n_active) {
    count_launches(5);
    const size_t Vh = (size_t)g->geom.V / 2;
    EpiStore<Rs, T::PS> es{w.tes.p, Vh, 0, RedSlots{nullptr, nullptr}};
    EventPair ev[5];
    TSM_TRY(ev[0].begin(s));
    launch_dslash_eo_tc<Rs, -1, T::PS, T::PLs>(w.nr_s, step_a(g, T::PLs, w.p.p, kappa, mup, nrhs), es, s);
    TSM_TRY(ev[0].end(s));
    TSM_TRY(ev[1].begin(s));
    {
      EpiMp<Rs, T::PS> e{w.q.p, Vh, w.st.as<RhsState>(), slots(w)};
      launch_dslash_eo_tc<Rs, -1, T::PS, T::PLs>(w.nr_s, step_b(g, T::PLs, w.tes.p, w.p.p, kappa, mup, nrhs), e, s);
    }
    TSM_TRY(ev[1].end(s));
    TSM_TRY(ev[2].begin(s));
    launch_dslash_eo_tc<Rs, +1, T::PS, T::PLs>(w.nr_s, step_a(g, T::PLs, w.q.p, kappa, -mup, nrhs), es, s);
    TSM_TRY(ev[2].end(s));
    TSM_TRY(ev[3].begin(s));
    {
      EpiCG<Rs, T::PA, T::PS> e{w.r.p, w.x.p, w.p.p, Vh, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash_eo_tc<Rs, +1, T::PS, T::PLs>(w.nr_s, step_b(g, T::PLs, w.tes.p, w.q.p, kappa, -mup, nrhs), e, s);
    }
    TSM_TRY(ev[3].end(s));
    TSM_TRY(ev[4].begin(s));
    dim3 eg(((int)Vh + EW_BS - 1) / EW_BS, nrhs);
    k_pupdate<T::PA, T::PS><<<eg, EW_BS, 0, s>>>(w.r.p, w.p.p, w.st.as<RhsState>(), 0, (int)Vh);
    TSM_TRY(ev[4].end(s));
    TSM_CUDA(cudaGetLastError());
    const double vf = (double)g->geom.V, vh = (double)Vh, n = (double)n_active;
    const double ls = link_site_bytes(T::PLs), bs = spinor_site_bytes(T::PS), ba = spinor_site_bytes(T::PA);
    const double fl = vh * n * (1392.0 + 96.0);  // hop + the two-term combination
    char name[48];
    snprintf(name, sizeof(name), "eo_hop_to_even_%s", pname());
    prof_add(name, ev[0].seconds(), vf * ls + n * vh * 2 * bs, fl);
    prof_add(name, ev[2].seconds(), vf * ls + n * vh * 2 * bs, fl);
    snprintf(name, sizeof(name), "eo_hop_to_odd_Mp_%s", pname());
    prof_add(name, ev[1].seconds(), vf * ls + n * vh * 3 * bs, fl + vh * n * 48.0);
    snprintf(name, sizeof(name), "eo_hop_to_odd_MdagQ_update_%s", pname());
    prof_add(name, ev[3].seconds(), vf * ls + n * vh * (3 * bs + 4 * ba), fl + vh * n * (96.0 + 48.0));
    snprintf(name, sizeof(name), "eo_p_update_%s", pname());
    prof_add(name, ev[4].seconds(), vh * n * (ba + 2 * bs), vh * n * 72.0);
    return TSM_OK;
  }

  // The graph of one chunk of iterations for (nrhs, kappa, mu'), captured on
  // stream s if not cached.  The kernels' arguments hold only workspace
  // pointers, kappa, mu' and solver constants; everything a solve changes
  // (rho, max_iter, the iterates) lives in the device state, so a cached graph
  // serves every later solve of that shape.
  static int ensure_graph(const tsm_gauge* g, EoWorkspace& w, int nrhs, double kappa, double mup,
                          const SolveParams& prm, cudaStream_t s, cudaGraphExec_t* out) {
    if (w.graph_kappa != kappa || w.graph_mup != mup) {
      for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
      w.graphs.clear();
      w.graph_kappa = kappa;
      w.graph_mup = mup;
    }
    auto found = w.graphs.find(nrhs);
    if (found == w.graphs.end()) {
      const int k = eo_chunk();
      cudaGraph_t graph;
      TSM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      for (int it = 0; it < k; ++it) iteration(g, w, nrhs, kappa, mup, prm, s);
      count_launches(-5LL * k);  // captured, not launched
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

  static int run_chunk(const tsm_gauge* g, EoWorkspace& w, int nrhs, double kappa, double mup, const SolveParams& prm,
                       cudaStream_t s) {
    cudaGraphExec_t exec;
    TSM_TRY(ensure_graph(g, w, nrhs, kappa, mup, prm, s, &exec));
    TSM_CUDA(cudaGraphLaunch(exec, s));
    count_launches(5LL * eo_chunk());
    return TSM_OK;
  }

  static void set_shapes(EoWorkspace& w) {
    const int nr_s = eo_nr(T::PS), nr_p = eo_nr(T::PP);
    if (nr_s != w.nr_s) {  // captured graphs bake in the launch shape
      for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
      w.graphs.clear();
    }
    w.nr_s = nr_s;
    w.nr_p = nr_p;
  }

  // r = b - Mhat^dag Mhat x_true for the masked right-hand sides (precise operator)
  static int replace_residual(const tsm_gauge* g, EoWorkspace& w, int nrhs, double kappa, double mup,
                              const SolveParams& prm, cudaStream_t s) {
    const size_t Vh = (size_t)g->geom.V / 2;
    dim3 eg(((int)Vh + EW_BS - 1) / EW_BS, nrhs);
    const void* xs = w.x.p;
    count_launches(T::XACC ? 6 : 5);
    if (T::XACC) {
      k_fold<T::PA, T::PXA><<<eg, EW_BS, 0, s>>>(w.x.p, w.xacc.p, w.mask.as<int>(), (int)Vh);
      xs = w.xacc.p;
    }
    const int* m = w.mask.as<int>();
    EpiStoreMasked<Rp, T::PP> to_tep{w.tep.p, Vh, m, RedSlots{nullptr, nullptr}};
    EpiStoreMasked<Rp, T::PP> to_t1{w.t1.p, Vh, m, RedSlots{nullptr, nullptr}};
    launch_dslash_eo<Rp, -1, T::PX, T::PLp>(w.nr_p, step_a(g, T::PLp, xs, kappa, mup, nrhs), to_tep, s);
    launch_dslash_eo<Rp, -1, T::PP, T::PLp>(w.nr_p, step_b(g, T::PLp, w.tep.p, xs, kappa, mup, nrhs), to_t1, s);
    launch_dslash_eo<Rp, +1, T::PP, T::PLp>(w.nr_p, step_a(g, T::PLp, w.t1.p, kappa, -mup, nrhs), to_tep, s);
    {
      EpiResidual<Rp, T::PP, T::PA> e{w.b.p, w.r.p, Vh, m, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash_eo<Rp, +1, T::PP, T::PLp>(w.nr_p, step_b(g, T::PLp, w.tep.p, w.t1.p, kappa, -mup, nrhs), e, s);
    }
    k_pupdate<T::PA, T::PS><<<eg, EW_BS, 0, s>>>(w.r.p, w.p.p, w.st.as<RhsState>(), 1, (int)Vh);
    TSM_CUDA(cudaGetLastError());
    return TSM_OK;
  }

  // eta split by parity (precise precision): eta_e, t1 = eta_o and
  // tep = M_ee^{-1} eta_e (split_sources)
  static int solve(tsm_gauge* g, EoWorkspace& w, int nrhs, double kappa, double mu, double rho, int max_iter,
                   int out_prec, void* x_out, int gamma5_out, tsm_solve_stats* stats, cudaStream_t s) {
    const double mup = 2.0 * kappa * mu;
    const double d = 1.0 + mup * mup;
    const SolveParams prm = params(g, rho, max_iter);
    const int V = g->geom.V;
    const size_t Vh = (size_t)V / 2;
    dim3 fg((V + EW_BS - 1) / EW_BS, nrhs), eg(((int)Vh + EW_BS - 1) / EW_BS, nrhs);
    set_shapes(w);
    count_launches(4);
    {  // t1 = eta_o - M_oe M_ee^{-1} eta_e = eta_o + kappa H tep   (in place on t1)
      EpiStore<Rp, T::PP> e{w.t1.p, Vh, 0, RedSlots{nullptr, nullptr}};
      launch_dslash_eo<Rp, -1, T::PP, T::PLp>(w.nr_p, args(g, T::PLp, w.tep.p, w.t1.p, 1, kappa, 1.0, 0.0, kappa, 0.0, nrhs),
                                              e, s);
    }
    {  // b = Mhat^dag t1, state initialisation
      EpiStore<Rp, T::PP> e{w.tep.p, Vh, 0, RedSlots{nullptr, nullptr}};
      launch_dslash_eo<Rp, +1, T::PP, T::PLp>(w.nr_p, step_a(g, T::PLp, w.t1.p, kappa, -mup, nrhs), e, s);
      EpiInitB<Rp, T::PP> ei{w.b.p, Vh, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash_eo<Rp, +1, T::PP, T::PLp>(w.nr_p, step_b(g, T::PLp, w.tep.p, w.t1.p, kappa, -mup, nrhs), ei, s);
    }
    k_init<T::PP, T::PA, T::PS, T::XACC, T::PXA>
        <<<eg, EW_BS, 0, s>>>(w.b.p, w.r.p, w.x.p, w.p.p, w.xacc.p, w.st.as<RhsState>(), (int)Vh);
    TSM_CUDA(cudaGetLastError());
    const long long limit = (long long)max_iter / eo_chunk() + 64;
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
      if (round > limit) return fail(TSM_ERR_CUDA, "even-odd solver exceeded its chunk bound");
      if (profiling()) {
        int n_active = 0;
        for (int r = 0; r < nrhs; ++r) n_active += (w.h_st[r].active != 0);
        TSM_TRY(iteration_profiled(g, w, nrhs, kappa, mup, prm, s, n_active));
      } else {
        TSM_TRY(run_chunk(g, w, nrhs, kappa, mup, prm, s));
      }
    }
    // s_o = x (+ xacc) into t1; s_e = M_ee^{-1} (eta_e + kappa H s_o) into tep; scatter
    count_launches(3);
    k_output<T::PA, T::PP, T::XACC, T::PXA><<<eg, EW_BS, 0, s>>>(w.x.p, w.xacc.p, w.t1.p, 0, (int)Vh);
    {
      EpiStore<Rp, T::PP> e{w.tep.p, Vh, 0, RedSlots{nullptr, nullptr}};
      launch_dslash_eo<Rp, -1, T::PP, T::PLp>(w.nr_p, 
          args(g, T::PLp, w.t1.p, w.eta_e.p, 0, kappa, 1.0 / d, -mup / d, kappa / d, -kappa * mup / d, nrhs), e, s);
    }
    switch (out_prec) {
      case TSM_F64:
        k_scatter_eo<TSM_F64, T::PP><<<fg, EW_BS, 0, s>>>(x_out, w.tep.p, w.t1.p, g->geom, gamma5_out);
        break;
      case TSM_F32:
        k_scatter_eo<TSM_F32, T::PP><<<fg, EW_BS, 0, s>>>(x_out, w.tep.p, w.t1.p, g->geom, gamma5_out);
        break;
      case TSM_F16:
        k_scatter_eo<TSM_F16, T::PP><<<fg, EW_BS, 0, s>>>(x_out, w.tep.p, w.t1.p, g->geom, gamma5_out);
        break;
      case TSM_BF16:
        k_scatter_eo<TSM_BF16, T::PP><<<fg, EW_BS, 0, s>>>(x_out, w.tep.p, w.t1.p, g->geom, gamma5_out);
        break;
      default: return fail(TSM_ERR_INVALID_ARG, "bad output precision %d", out_prec);
    }
    TSM_CUDA(cudaGetLastError());
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
int solve_eo_kind(tsm_gauge* g, double kappa, double mu, double rho, int max_iter, int nrhs, const void* eta,
                  int eta_prec, uint64_t seed, uint64_t first, int out_prec, void* x_out, int gamma5_io,
                  tsm_solve_stats* stats, cudaStream_t s, int slot) {
  using T = Traits<KIND>;
  EoWorkspace* wp;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    auto& ws = g->eo_ws[KIND + 64 * slot];
    if (!ws) ws.reset(new EoWorkspace());
    wp = ws.get();
  }
  EoWorkspace& w = *wp;
  std::lock_guard<std::mutex> wlock(w.mu);
  TSM_TRY(w.order.enter(s));
  TSM_TRY(SolverEO<KIND>::reserve(g, w, nrhs, s));
  // the source split by parity: eta_e, t1 = eta_o, tep = M_ee^{-1} eta_e
  const double mup = 2.0 * kappa * mu, d = 1.0 + mup * mup;
  if (eta) {
    TSM_TRY(spinor_convert(g, T::PP, w.full.p, eta_prec, eta, nrhs, gamma5_io, s));
    dim3 fg((g->geom.V + EW_BS - 1) / EW_BS, nrhs);
    count_launches(1);
    k_split_eo<T::PP><<<fg, EW_BS, 0, s>>>(w.full.p, w.eta_e.p, w.t1.p, w.tep.p, 1.0 / d, -mup / d, g->geom);
    TSM_CUDA(cudaGetLastError());
  } else {
    TSM_TRY(make_sources_eo(g, seed, first, nrhs, T::PP, w.eta_e.p, w.t1.p, w.tep.p, 1.0 / d, -mup / d, s));
  }
  const int rc = SolverEO<KIND>::solve(g, w, nrhs, kappa, mu, rho, max_iter, out_prec, x_out, gamma5_io, stats, s);
  const int rc_order = w.order.leave(s);
  return rc != TSM_OK ? rc : rc_order;
}

}  // namespace

namespace {

DslashArgs eo_args(const tsm_gauge* g, int prec, const void* in, const void* ctr, int par, double kappa, double c0,
                   double c1, double h0, double h1, int nrhs) {
  DslashArgs a;
  a.g = g->geom;
  a.links = g->links[prec].p;
  a.in = in;
  a.nrhs = nrhs;
  a.nblk = (g->geom.V / 2 + DSLASH_BS - 1) / DSLASH_BS;
  set_coeffs(a, kappa, 0.0);
  set_eo(a, ctr, par, c0, c1, h0, h1);
  return a;
}

// out_o = Mhat in_o (dag: Mhat^dag) on half-volume fields; t_e is scratch
template <typename R, int P, int SF>
void mhat_launch(const tsm_gauge* g, double kappa, double tau, const void* in_o, void* t_e, void* out_o, int nrhs,
                 cudaStream_t s) {
  const size_t Vh = (size_t)g->geom.V / 2;
  const double d = 1.0 + tau * tau;
  EpiStore<R, P> et{t_e, Vh, 0, RedSlots{nullptr, nullptr}};
  EpiStore<R, P> eo{out_o, Vh, 0, RedSlots{nullptr, nullptr}};
  launch_dslash_eo_tc<R, SF, P, P>(1, eo_args(g, P, in_o, nullptr, 0, kappa, 0.0, 0.0, -kappa / d, kappa * tau / d, nrhs),
                                et, s);
  launch_dslash_eo_tc<R, SF, P, P>(1, eo_args(g, P, t_e, in_o, 1, kappa, 1.0, tau, kappa, 0.0, nrhs), eo, s);
}

template <typename R, int P>
int mhat_apply(tsm_gauge* g, int dag, double kappa, double mu, const void* in, void* out, int nrhs, cudaStream_t s) {
  const int V = g->geom.V;
  const size_t half = (size_t)nrhs * spinor_chunks(P) * (size_t)(V / 2) * 16;
  ScratchLease lease(g->eo_tmp);
  TSM_TRY(lease.acquire(3 * half, s));
  char* base = static_cast<char*>(lease.ptr());
  void *in_o = base, *t_e = base + half, *out_o = base + 2 * half;
  const double mup = 2.0 * kappa * mu;
  dim3 fg((V + EW_BS - 1) / EW_BS, nrhs);
  count_launches(5);
  k_gather_eo<P><<<fg, EW_BS, 0, s>>>(in, t_e, in_o, g->geom);  // the even half lands in scratch
  if (dag)
    mhat_launch<R, P, +1>(g, kappa, -mup, in_o, t_e, out_o, nrhs, s);
  else
    mhat_launch<R, P, -1>(g, kappa, mup, in_o, t_e, out_o, nrhs, s);
  TSM_CUDA(cudaMemsetAsync(t_e, 0, half, s));  // zeros on the even sites of the result
  k_scatter_eo<P, P><<<fg, EW_BS, 0, s>>>(out, t_e, out_o, g->geom, 0);
  TSM_CUDA(cudaGetLastError());
  return lease.release(s);
}

}  // namespace

int schur_apply(tsm_gauge* g, int prec, int dag, double kappa, double mu, const void* in, void* out, int nrhs,
                cudaStream_t s) {
  if (!eo_lattice(g->geom)) return fail(TSM_ERR_INVALID_ARG, "the Schur operator needs even extents");
  switch (prec) {
    case TSM_F64: return mhat_apply<double, TSM_F64>(g, dag, kappa, mu, in, out, nrhs, s);
    case TSM_F32: return mhat_apply<float, TSM_F32>(g, dag, kappa, mu, in, out, nrhs, s);
    case TSM_F16: return mhat_apply<float, TSM_F16>(g, dag, kappa, mu, in, out, nrhs, s);
    case TSM_BF16: return mhat_apply<float, TSM_BF16>(g, dag, kappa, mu, in, out, nrhs, s);
  }
  return fail(TSM_ERR_INVALID_ARG, "bad precision %d", prec);
}

namespace {
template <int KIND>
int prepare_eo_kind(tsm_gauge* g, int nrhs, double kappa, double mu, int slot, cudaStream_t s) {
  EoWorkspace* wp;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    auto& ws = g->eo_ws[KIND + 64 * slot];
    if (!ws) ws.reset(new EoWorkspace());
    wp = ws.get();
  }
  EoWorkspace& w = *wp;
  std::lock_guard<std::mutex> wlock(w.mu);
  TSM_TRY(w.order.enter(s));
  TSM_TRY(SolverEO<KIND>::reserve(g, w, nrhs, s));
  if (!profiling()) {  // the chunk graph too: a solve then captures nothing
    SolverEO<KIND>::set_shapes(w);
    cudaGraphExec_t exec;
    TSM_TRY(SolverEO<KIND>::ensure_graph(g, w, nrhs, kappa, 2.0 * kappa * mu, SolverEO<KIND>::params(g, 0.5, 1), s,
                                         &exec));
  }
  return w.order.leave(s);
}
}  // namespace

// Workspace and chunk graph of an even-odd solve of nrhs right-hand sides at
// (kappa, mu) on `slot`, made ahead of the solve (the checkerboarded stencils
// are not autotuned).
int prepare_eo(tsm_gauge* g, int solver, int nrhs, double kappa, double mu, int slot, cudaStream_t s) {
  if (!eo_lattice(g->geom)) return fail(TSM_ERR_INVALID_ARG, "even-odd solves need even extents");
  switch (solver & ~TSM_SOLVER_EO) {
    case TSM_SOLVER_F64: return prepare_eo_kind<TSM_SOLVER_F64>(g, nrhs, kappa, mu, slot, s);
    case TSM_SOLVER_F32_RELIABLE: return prepare_eo_kind<TSM_SOLVER_F32_RELIABLE>(g, nrhs, kappa, mu, slot, s);
    case TSM_SOLVER_LP_F16: return prepare_eo_kind<TSM_SOLVER_LP_F16>(g, nrhs, kappa, mu, slot, s);
    case TSM_SOLVER_LP_BF16: return prepare_eo_kind<TSM_SOLVER_LP_BF16>(g, nrhs, kappa, mu, slot, s);
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown solver %d", solver);
}

int solve_batch_eo(tsm_gauge* g, double kappa, double mu, int solver, double rho, int max_iter, int nrhs,
                   const void* eta, int eta_prec, uint64_t seed, uint64_t first, int out_prec, void* x_out,
                   int gamma5_io, tsm_solve_stats* stats, cudaStream_t s, int slot) {
  if (!eo_lattice(g->geom)) return fail(TSM_ERR_INVALID_ARG, "even-odd solves need even extents");
  switch (solver & ~TSM_SOLVER_EO) {
    case TSM_SOLVER_F64:
      return solve_eo_kind<TSM_SOLVER_F64>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first, out_prec,
                                           x_out, gamma5_io, stats, s, slot);
    case TSM_SOLVER_F32_RELIABLE:
      return solve_eo_kind<TSM_SOLVER_F32_RELIABLE>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                                    out_prec, x_out, gamma5_io, stats, s, slot);
    case TSM_SOLVER_LP_F16:
      return solve_eo_kind<TSM_SOLVER_LP_F16>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                              out_prec, x_out, gamma5_io, stats, s, slot);
    case TSM_SOLVER_LP_BF16:
      return solve_eo_kind<TSM_SOLVER_LP_BF16>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                               out_prec, x_out, gamma5_io, stats, s, slot);
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown solver %d", solver);
}

}  // namespace tsm
