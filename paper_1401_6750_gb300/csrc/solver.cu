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

namespace tsm {

namespace {

constexpr int EW_BS = 256;

struct SolveParams {
  double rho2;
  double delta2;
  double inv_ncomp;  // 1 / (12 V)
  int max_iter;
  int scaled;
};

template <int KIND>
struct Traits;
template <>
struct Traits<TSM_SOLVER_F64> {
  using Rs = double;
  using Rp = double;
  static constexpr int PS = TSM_F64, PA = TSM_F64, PP = TSM_F64, PLs = TSM_F64, PLp = TSM_F64, PX = TSM_F64;
  static constexpr bool XACC = false, SCALED = false;
  static constexpr double DELTA = 0.0;
};
template <>
struct Traits<TSM_SOLVER_F32_RELIABLE> {
  using Rs = float;
  using Rp = double;
  static constexpr int PS = TSM_F32, PA = TSM_F32, PP = TSM_F64, PLs = TSM_F32, PLp = TSM_F64, PX = TSM_F64;
  static constexpr bool XACC = true, SCALED = false;
  // FP32 recurrences stay accurate over three decades below the last true residual
  static constexpr double DELTA = 1e-3;
};
template <>
struct Traits<TSM_SOLVER_LP_F16> {
  using Rs = float;
  using Rp = float;
  static constexpr int PS = TSM_F16, PA = TSM_F32, PP = TSM_F32, PLs = TSM_F16, PLp = TSM_F32, PX = TSM_F32;
  static constexpr bool XACC = false, SCALED = true;
  static constexpr double DELTA = 0.1;
};
template <>
struct Traits<TSM_SOLVER_LP_BF16> {
  using Rs = float;
  using Rp = float;
  static constexpr int PS = TSM_BF16, PA = TSM_F32, PP = TSM_F32, PLs = TSM_BF16, PLp = TSM_F32, PX = TSM_F32;
  static constexpr bool XACC = false, SCALED = true;
  static constexpr double DELTA = 0.1;
};

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// ---------------------------------------------------------------- epilogues
// b = M^dag eta; |b|^2 initialises the state of each right-hand side.
template <typename R, int PO>
struct EpiInitB {
  static constexpr bool kReduce = true;
  void* out;
  size_t V;
  RhsState* st;
  RedSlots red;
  SolveParams prm;
  __device__ bool active(int) const { return true; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    SpinorIO<PO>::store(out, V, rhs, i, o);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) n += norm2(o[k]);
    return n;
  }
  __device__ void finalize(int rhs, double bb) const {
    RhsState& s = st[rhs];
    s.bb = bb;
    s.rho2bb = prm.rho2 * bb;
    s.rr = bb;
    s.r_max2 = bb;
    s.true_rr = bb;
    s.delta2 = prm.delta2;
    s.alpha = s.beta = 0.0;
    s.sigma = (prm.scaled && bb > 0.0) ? sqrt(bb * prm.inv_ncomp) : 1.0;
    s.c_r = 1.0 / s.sigma;
    s.c_p = 0.0;
    s.iter = 0;
    s.max_iter = prm.max_iter;
    s.need_ru = 0;
    s.n_ru = 0;
    s.restarts = 0;
    s.restart_p = 0;
    if (!finite_d(bb)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
    } else if (bb == 0.0) {
      s.status = ST_DONE;
      s.active = 0;
    } else {
      s.status = ST_RUNNING;
      s.active = 1;
    }
  }
};

// q = M p (sloppy), |q|^2 -> alpha.
template <typename R, int PQ>
struct EpiMp {
  static constexpr bool kReduce = true;
  void* q;
  size_t V;
  RhsState* st;
  RedSlots red;
  __device__ bool active(int rhs) const { return st[rhs].active != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    SpinorIO<PQ>::store(q, V, rhs, i, o);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) n += norm2(o[k]);
    return n;
  }
  __device__ void finalize(int rhs, double qq) const {
    RhsState& s = st[rhs];
    s.restart_p = 0;
    const double pap = s.sigma * s.sigma * qq;
    if (!(pap > 0.0) || !finite_d(pap)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
      return;
    }
    s.alpha = s.rr / pap;
  }
};

// Ap = M^dag q (sloppy); r -= alpha Ap; x += alpha p; |r|^2 -> beta, stop test.
template <typename R, int PA, int PS>
struct EpiCG {
  static constexpr bool kReduce = true;
  void* r;
  void* x;
  const void* p;
  size_t V;
  RhsState* st;
  RedSlots red;
  SolveParams prm;
  __device__ bool active(int rhs) const { return st[rhs].active != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&ap)[12]) const {
    const R a = (R)(st[rhs].alpha * st[rhs].sigma);
    cplx<R> rv[12], xv[12], pv[12];
    SpinorIO<PA>::load(r, V, rhs, i, rv);
    SpinorIO<PA>::load(x, V, rhs, i, xv);
    SpinorIO<PS>::load(p, V, rhs, i, pv);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k] = rv[k] - a * ap[k];
      xv[k] = xv[k] + a * pv[k];
      n += norm2(rv[k]);
    }
    SpinorIO<PA>::store(r, V, rhs, i, rv);
    SpinorIO<PA>::store(x, V, rhs, i, xv);
    return n;
  }
  __device__ void finalize(int rhs, double rr_new) const {
    RhsState& s = st[rhs];
    s.iter += 1;
    if (!finite_d(rr_new)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
      return;
    }
    const double beta = rr_new / s.rr;
    s.beta = beta;
    s.rr = rr_new;
    if (rr_new > s.r_max2) s.r_max2 = rr_new;
    double sig = 1.0;
    if (prm.scaled) {
      sig = sqrt(rr_new * prm.inv_ncomp);
      if (!(sig > 0.0)) sig = 1.0;
    }
    s.c_r = 1.0 / sig;
    s.c_p = beta * s.sigma / sig;
    s.sigma = sig;
    if (rr_new <= s.rho2bb) {
      s.status = ST_ITER_CONV;
      s.active = 0;
    } else if (s.iter >= s.max_iter) {
      s.status = ST_MAXITER;
      s.active = 0;
    } else if (s.delta2 > 0.0 && rr_new < s.delta2 * s.r_max2) {
      s.need_ru = 1;
    }
  }
};

// t = M x with the precise operator, for the rhs in mask.
template <typename R, int PO>
struct EpiStoreMasked {
  static constexpr bool kReduce = false;
  void* out;
  size_t V;
  const int* mask;
  RedSlots red;
  __device__ bool active(int rhs) const { return mask[rhs] != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    SpinorIO<PO>::store(out, V, rhs, i, o);
    return (R)0;
  }
  __device__ void finalize(int, double) const {}
};

// r = b - M^dag t (precise); |r|^2 is the true residual.
template <typename R, int PB, int PA>
struct EpiResidual {
  static constexpr bool kReduce = true;
  const void* b;
  void* r;
  size_t V;
  const int* mask;
  RhsState* st;
  RedSlots red;
  SolveParams prm;
  __device__ bool active(int rhs) const { return mask[rhs] != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    cplx<R> bv[12];
    SpinorIO<PB>::load(b, V, rhs, i, bv);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      bv[k] = bv[k] - o[k];
      n += norm2(bv[k]);
    }
    SpinorIO<PA>::store(r, V, rhs, i, bv);
    return n;
  }
  __device__ void finalize(int rhs, double rr) const {
    RhsState& s = st[rhs];
    s.true_rr = rr;
    s.rr = rr;
    s.r_max2 = rr;
    s.need_ru = 0;
    s.n_ru += 1;
    if (!finite_d(rr)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
      return;
    }
    if (s.status == ST_ITER_CONV || s.status == ST_MAXITER) {
      if (rr <= s.rho2bb) {
        s.status = ST_DONE;
        s.active = 0;
      } else if (s.status == ST_MAXITER || s.iter >= s.max_iter) {
        s.status = ST_FAILED;
        s.active = 0;
      } else {
        // restart from the true residual: p = r
        s.status = ST_RUNNING;
        s.active = 1;
        s.restarts += 1;
        s.restart_p = 1;
        double sig = 1.0;
        if (prm.scaled) {
          sig = sqrt(rr * prm.inv_ncomp);
          if (!(sig > 0.0)) sig = 1.0;
        }
        s.c_r = 1.0 / sig;
        s.c_p = 0.0;
        s.sigma = sig;
      }
    }
  }
};

// ---------------------------------------------------------------- elementwise kernels
template <int PB, int PA, int PS, bool XACC>
__global__ void k_init(const void* b, void* r, void* x, void* p, double2* xacc, const RhsState* st, int V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= V) return;
  cplx<double> v[12], z[12];
  SpinorIO<PB>::load(b, (size_t)V, rhs, i, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = mk<double>(0.0, 0.0);
  SpinorIO<PA>::store(r, (size_t)V, rhs, i, v);
  SpinorIO<PA>::store(x, (size_t)V, rhs, i, z);
  if (XACC) SpinorIO<TSM_F64>::store(xacc, (size_t)V, rhs, i, z);
  const double c = st[rhs].c_r;
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = c * v[k];
  SpinorIO<PS>::store(p, (size_t)V, rhs, i, v);
}

// p = c_r r + c_p p for rhs with (mode 0) active or (mode 1) restart_p set.
template <int PA, int PS>
__global__ void k_pupdate(const void* r, void* p, const RhsState* st, int mode, int V) {
  const int rhs = blockIdx.y;
  const RhsState& s = st[rhs];
  if (mode == 0 ? !s.active : !s.restart_p) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const float cr = (float)s.c_r, cp = (float)s.c_p;
  cplx<float> rv[12], pv[12];
  SpinorIO<PA>::load(r, (size_t)V, rhs, i, rv);
  SpinorIO<PS>::load(p, (size_t)V, rhs, i, pv);
#pragma unroll
  for (int k = 0; k < 12; ++k) pv[k] = cr * rv[k] + cp * pv[k];
  SpinorIO<PS>::store(p, (size_t)V, rhs, i, pv);
}

// FP64 variant for the all-FP64 solver (coefficients kept in double).
template <>
__global__ void k_pupdate<TSM_F64, TSM_F64>(const void* r, void* p, const RhsState* st, int mode, int V) {
  const int rhs = blockIdx.y;
  const RhsState& s = st[rhs];
  if (mode == 0 ? !s.active : !s.restart_p) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const double cr = s.c_r, cp = s.c_p;
  cplx<double> rv[12], pv[12];
  SpinorIO<TSM_F64>::load(r, (size_t)V, rhs, i, rv);
  SpinorIO<TSM_F64>::load(p, (size_t)V, rhs, i, pv);
#pragma unroll
  for (int k = 0; k < 12; ++k) pv[k] = cr * rv[k] + cp * pv[k];
  SpinorIO<TSM_F64>::store(p, (size_t)V, rhs, i, pv);
}

// xacc += x; x = 0 (masked): fold the sloppy solution into the FP64 accumulator.
template <int PA>
__global__ void k_fold(void* x, double2* xacc, const int* mask, int V) {
  const int rhs = blockIdx.y;
  if (!mask[rhs]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  cplx<double> xv[12], av[12];
  SpinorIO<PA>::load(x, (size_t)V, rhs, i, xv);
  SpinorIO<TSM_F64>::load(xacc, (size_t)V, rhs, i, av);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    av[k] = av[k] + xv[k];
    xv[k] = mk<double>(0.0, 0.0);
  }
  SpinorIO<TSM_F64>::store(xacc, (size_t)V, rhs, i, av);
  SpinorIO<PA>::store(x, (size_t)V, rhs, i, xv);
}

template <int PA, int PO, bool XACC>
__global__ void k_output(const void* x, const double2* xacc, void* out, int gamma5, int V) {
  const int rhs = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  cplx<double> v[12];
  SpinorIO<PA>::load(x, (size_t)V, rhs, i, v);
  if (XACC) {
    cplx<double> a[12];
    SpinorIO<TSM_F64>::load(xacc, (size_t)V, rhs, i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = v[k] + a[k];
  }
  if (gamma5) {
#pragma unroll
    for (int k = 6; k < 12; ++k) v[k] = mk<double>(-v[k].re, -v[k].im);
  }
  SpinorIO<PO>::store(out, (size_t)V, rhs, i, v);
}

size_t field_bytes(int prec, int V, int nrhs) { return (size_t)nrhs * spinor_chunks(prec) * (size_t)V * 16; }

}  // namespace

// ---------------------------------------------------------------- workspace
struct SolverWorkspace {
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
  return (solver == TSM_SOLVER_F64 || solver == TSM_SOLVER_F32_RELIABLE) ? TSM_F64 : TSM_F32;
}
int solver_output_prec(int solver) {
  return (solver == TSM_SOLVER_F64 || solver == TSM_SOLVER_F32_RELIABLE) ? TSM_F64 : TSM_F32;
}
unsigned solver_link_precs(int solver) {
  switch (solver) {
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

  static int reserve(tsm_gauge* g, SolverWorkspace& w, int nrhs) {
    if (w.cap >= nrhs) return TSM_OK;
    for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
    w.graphs.clear();
    const int V = g->geom.V;
    w.nblk = (V + DSLASH_BS - 1) / DSLASH_BS;
    TSM_TRY(w.st.reserve(sizeof(RhsState) * nrhs));
    TSM_TRY(w.partial.reserve(sizeof(double) * (size_t)nrhs * w.nblk));
    TSM_TRY(w.counter.reserve(sizeof(unsigned) * nrhs));
    TSM_CUDA(cudaMemset(w.counter.p, 0, sizeof(unsigned) * nrhs));
    TSM_TRY(w.mask.reserve(sizeof(int) * nrhs));
    TSM_TRY(w.b.reserve(field_bytes(T::PP, V, nrhs)));
    TSM_TRY(w.t.reserve(field_bytes(T::PP, V, nrhs)));
    TSM_TRY(w.x.reserve(field_bytes(T::PA, V, nrhs)));
    TSM_TRY(w.r.reserve(field_bytes(T::PA, V, nrhs)));
    TSM_TRY(w.p.reserve(field_bytes(T::PS, V, nrhs)));
    TSM_TRY(w.q.reserve(field_bytes(T::PS, V, nrhs)));
    if (T::XACC) TSM_TRY(w.xacc.reserve(field_bytes(TSM_F64, V, nrhs)));
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
    a.kappa = kappa;
    a.tw = tw;
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
    p.rho2 = rho * rho;
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
    // kernel arguments carry kappa and mu'; a change invalidates the cached graphs
    if (w.graph_kappa != kappa || w.graph_mup != mup) {
      for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
      w.graphs.clear();
      w.graph_kappa = kappa;
      w.graph_mup = mup;
    }
    auto found = w.graphs.find(nrhs);
    if (found == w.graphs.end()) {
      cudaGraph_t graph;
      TSM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      for (int i = 0; i < k; ++i) iteration(g, w, nrhs, kappa, mup, prm, s);
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      cudaGraphExec_t exec;
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      found = w.graphs.emplace(nrhs, exec).first;
    }
    TSM_CUDA(cudaGraphLaunch(found->second, s));
    count_launches(3LL * k);
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
      k_fold<T::PA><<<eg, EW_BS, 0, s>>>(w.x.p, w.xacc.as<double2>(), w.mask.as<int>(), g->geom.V);
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
    {
      int nr_s = 1, nr_p = 1;
      TSM_TRY(tuned_nr(g, T::PS, T::PLs, nrhs, s, &nr_s));
      TSM_TRY(tuned_nr(g, T::PP, T::PLp, nrhs, s, &nr_p));
      if (nr_s != w.nr_s) {  // captured graphs bake in the launch shape
        for (auto& kv : w.graphs) cudaGraphExecDestroy(kv.second);
        w.graphs.clear();
      }
      w.nr_s = nr_s;
      w.nr_p = nr_p;
    }
    dim3 eg((g->geom.V + EW_BS - 1) / EW_BS, nrhs);
    // b = M^dag eta (precise), state initialisation
    count_launches(2);
    {
      EpiInitB<Rp, T::PP> e{w.b.p, V, w.st.as<RhsState>(), slots(w), prm};
      launch_dslash<Rp, +1, T::PP, T::PLp>(w.nr_p, args(g, T::PLp, w.t.p, kappa, -mup, nrhs), e, s);
    }
    k_init<T::PP, T::PA, T::PS, T::XACC>
        <<<eg, EW_BS, 0, s>>>(w.b.p, w.r.p, w.x.p, w.p.p, w.xacc.as<double2>(), w.st.as<RhsState>(), g->geom.V);
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
    k_output<T::PA, T::PP, T::XACC><<<eg, EW_BS, 0, s>>>(w.x.p, w.xacc.as<double2>(), w.t.p, gamma5_out,
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
               tsm_solve_stats* stats, cudaStream_t s) {
  using T = Traits<KIND>;
  std::lock_guard<std::mutex> lock(g->mu);
  auto& slot = g->solver_ws[KIND];
  if (!slot) slot.reset(new SolverWorkspace());
  SolverWorkspace& w = *slot;
  w.kind = KIND;
  TSM_TRY(Solver<KIND>::reserve(g, w, nrhs));
  if (eta) {
    TSM_TRY(spinor_convert(g, T::PP, w.t.p, eta_prec, eta, nrhs, gamma5_io, s));
  } else {
    TSM_TRY(make_sources(g, seed, first, nrhs, T::PP, w.t.p, s));
  }
  return Solver<KIND>::solve(g, w, nrhs, kappa, mu, rho, max_iter, out_prec, x_out, gamma5_io, stats, s);
}

}  // namespace

// eta == nullptr: Z4 sources (seed, first) are generated in place.
int solve_batch_impl(tsm_gauge* g, double kappa, double mu, int solver, double rho, int max_iter, int nrhs,
                     const void* eta, int eta_prec, uint64_t seed, uint64_t first, int out_prec, void* x_out,
                     int gamma5_io, tsm_solve_stats* stats, cudaStream_t s) {
  const unsigned need = solver_link_precs(solver);
  if ((g->precisions & need) != need)
    return fail(TSM_ERR_INVALID_ARG, "solver %d needs gauge copies 0x%x, gauge has 0x%x", solver, need,
                g->precisions);
  switch (solver) {
    case TSM_SOLVER_F64:
      return solve_kind<TSM_SOLVER_F64>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first, out_prec,
                                        x_out, gamma5_io, stats, s);
    case TSM_SOLVER_F32_RELIABLE:
      return solve_kind<TSM_SOLVER_F32_RELIABLE>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                                 out_prec, x_out, gamma5_io, stats, s);
    case TSM_SOLVER_LP_F16:
      return solve_kind<TSM_SOLVER_LP_F16>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                           out_prec, x_out, gamma5_io, stats, s);
    case TSM_SOLVER_LP_BF16:
      return solve_kind<TSM_SOLVER_LP_BF16>(g, kappa, mu, rho, max_iter, nrhs, eta, eta_prec, seed, first,
                                            out_prec, x_out, gamma5_io, stats, s);
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown solver %d", solver);
}

}  // namespace tsm
