// Uneven batches: several solve instances -- each its own gauge field
// (lattice size), twisted mass and set of Z4 sources -- advanced by ONE
// launch per CG kernel.  Each launch's blocks are partitioned by instance
// (a descriptor table gives every instance its geometry, links, vectors,
// per-right-hand-side states and reduction slots), so a small lattice fills
// the GPU next to a large one instead of in a launch of its own.  Every
// right-hand side keeps its own convergence flag; an instance is done when all
// of its right-hand sides are.  Per-right-hand-side arithmetic is that of the
// single-instance solver (same stencil, same fixed-order reductions over the
// instance's own blocks), so results equal solving each instance alone.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "dslash.cuh"
#include "internal.h"
#include "solver_kernels.cuh"

namespace tsm {

namespace {

using namespace solverk;

struct InstDesc {
  Geom g;
  const void* links_s;
  const void* links_p;
  double kappa, mup;
  double inv_ncomp;  // 1 / (12 V)
  int nrhs;
  int nblk;     // stencil blocks per right-hand side
  int dblock0;  // first stencil block of the instance in a multi launch
  int eblk;     // element-wise blocks per right-hand side
  int eblock0;  // first element-wise block
  void *b, *t, *x, *r, *p, *q;
  void* xacc;
  RhsState* st;
  double* partial;
  unsigned* counter;
  int* mask;
};

__device__ __forceinline__ int find_inst(const InstDesc* d, int n, int bid, bool elementwise) {
  int k = 0;
  while (k + 1 < n && bid >= (elementwise ? d[k + 1].eblock0 : d[k + 1].dblock0)) ++k;
  return k;
}

template <typename R, int SF, int PIN, int PL, class Maker>
__global__ void __launch_bounds__(DSLASH_BS) multi_dslash(const InstDesc* __restrict__ d, int n, Maker mk) {
  const int k = find_inst(d, n, blockIdx.x, false);
  const InstDesc& I = d[k];
  DslashArgs a;
  a.g = I.g;
  a.links = mk.links(I);
  a.in = mk.in(I);
  a.nblk = I.nblk;
  a.nrhs = I.nrhs;
  set_coeffs(a, I.kappa, mk.tw(I));
  dslash_block<R, SF, PIN, PL, 1>(a, mk.epi(I), blockIdx.x - I.dblock0);
}

template <class T, typename Rx>
struct MakeInitB {  // b = M^dag eta (precise)
  SolveParams prm;
  __device__ const void* links(const InstDesc& I) const { return I.links_p; }
  __device__ const void* in(const InstDesc& I) const { return I.t; }
  __device__ double tw(const InstDesc& I) const { return -I.mup; }
  __device__ EpiInitB<Rx, T::PP> epi(const InstDesc& I) const {
    SolveParams p = prm;
    p.inv_ncomp = I.inv_ncomp;
    return EpiInitB<Rx, T::PP>{I.b, (size_t)I.g.V, I.st, RedSlots{I.partial, I.counter}, p};
  }
};
template <class T, typename Rx>
struct MakeMp {  // q = M p (sloppy)
  __device__ const void* links(const InstDesc& I) const { return I.links_s; }
  __device__ const void* in(const InstDesc& I) const { return I.p; }
  __device__ double tw(const InstDesc& I) const { return I.mup; }
  __device__ EpiMp<Rx, T::PS> epi(const InstDesc& I) const {
    return EpiMp<Rx, T::PS>{I.q, (size_t)I.g.V, I.st, RedSlots{I.partial, I.counter}};
  }
};
template <class T, typename Rx>
struct MakeCG {  // Ap = M^dag q; r, x update
  SolveParams prm;
  __device__ const void* links(const InstDesc& I) const { return I.links_s; }
  __device__ const void* in(const InstDesc& I) const { return I.q; }
  __device__ double tw(const InstDesc& I) const { return -I.mup; }
  __device__ EpiCG<Rx, T::PA, T::PS> epi(const InstDesc& I) const {
    SolveParams p = prm;
    p.inv_ncomp = I.inv_ncomp;
    return EpiCG<Rx, T::PA, T::PS>{I.r, I.x, I.p, (size_t)I.g.V, I.st, RedSlots{I.partial, I.counter}, p};
  }
};
template <class T, typename Rx>
struct MakeRU1 {  // t = M x_true (precise, masked)
  __device__ const void* links(const InstDesc& I) const { return I.links_p; }
  __device__ const void* in(const InstDesc& I) const { return T::XACC ? (const void*)I.xacc : I.x; }
  __device__ double tw(const InstDesc& I) const { return I.mup; }
  __device__ EpiStoreMasked<Rx, T::PP> epi(const InstDesc& I) const {
    return EpiStoreMasked<Rx, T::PP>{I.t, (size_t)I.g.V, I.mask, RedSlots{nullptr, nullptr}};
  }
};
template <class T, typename Rx>
struct MakeRU2 {  // r = b - M^dag t (precise, masked), true residual
  SolveParams prm;
  __device__ const void* links(const InstDesc& I) const { return I.links_p; }
  __device__ const void* in(const InstDesc& I) const { return I.t; }
  __device__ double tw(const InstDesc& I) const { return -I.mup; }
  __device__ EpiResidual<Rx, T::PP, T::PA> epi(const InstDesc& I) const {
    SolveParams p = prm;
    p.inv_ncomp = I.inv_ncomp;
    return EpiResidual<Rx, T::PP, T::PA>{I.b, I.r, (size_t)I.g.V, I.mask, I.st, RedSlots{I.partial, I.counter}, p};
  }
};

// ---------------------------------------------------------------- element-wise, all instances
template <class T>
__global__ void multi_init(const InstDesc* __restrict__ d, int n) {
  const InstDesc& I = d[find_inst(d, n, blockIdx.x, true)];
  const int lb = blockIdx.x - I.eblock0, rhs = lb / I.eblk, i = (lb % I.eblk) * EW_BS + threadIdx.x;
  if (i >= I.g.V) return;
  const size_t V = (size_t)I.g.V;
  using R = ew_real<T::PP, T::PA, T::PS, (T::XACC ? T::PXA : T::PA)>;
  cplx<R> v[12], z[12];
  SpinorIO<T::PP>::load(I.b, V, rhs, i, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = mk<R>(0, 0);
  SpinorIO<T::PA>::store(I.r, V, rhs, i, v);
  SpinorIO<T::PA>::store(I.x, V, rhs, i, z);
  if (T::XACC) SpinorIO<T::PXA>::store(I.xacc, V, rhs, i, z);
  const R c = (R)I.st[rhs].c_r;
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = c * v[k];
  SpinorIO<T::PS>::store(I.p, V, rhs, i, v);
}

// p = c_r r + c_p p for right-hand sides that are active (mode 0) or restarting (mode 1)
template <class T>
__global__ void multi_pupdate(const InstDesc* __restrict__ d, int n, int mode) {
  const InstDesc& I = d[find_inst(d, n, blockIdx.x, true)];
  const int lb = blockIdx.x - I.eblock0, rhs = lb / I.eblk, i = (lb % I.eblk) * EW_BS + threadIdx.x;
  const RhsState& s = I.st[rhs];
  if (mode == 0 ? !s.active : !s.restart_p) return;
  if (i >= I.g.V) return;
  const size_t V = (size_t)I.g.V;
  using Rq = typename T::Rs;
  const Rq cr = (Rq)s.c_r, cp = (Rq)s.c_p;
  cplx<Rq> rv[12], pv[12];
  SpinorIO<T::PA>::load(I.r, V, rhs, i, rv);
  SpinorIO<T::PS>::load(I.p, V, rhs, i, pv);
#pragma unroll
  for (int k = 0; k < 12; ++k) pv[k] = cr * rv[k] + cp * pv[k];
  SpinorIO<T::PS>::store(I.p, V, rhs, i, pv);
}

template <class T>
__global__ void multi_fold(const InstDesc* __restrict__ d, int n) {
  const InstDesc& I = d[find_inst(d, n, blockIdx.x, true)];
  const int lb = blockIdx.x - I.eblock0, rhs = lb / I.eblk, i = (lb % I.eblk) * EW_BS + threadIdx.x;
  if (!I.mask[rhs] || i >= I.g.V) return;
  const size_t V = (size_t)I.g.V;
  using R = ew_real<T::PA, T::PXA>;
  cplx<R> xv[12], av[12];
  SpinorIO<T::PA>::load(I.x, V, rhs, i, xv);
  SpinorIO<T::PXA>::load(I.xacc, V, rhs, i, av);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    av[k] = av[k] + xv[k];
    xv[k] = mk<R>(0, 0);
  }
  SpinorIO<T::PXA>::store(I.xacc, V, rhs, i, av);
  SpinorIO<T::PA>::store(I.x, V, rhs, i, xv);
}

template <class T>
__global__ void multi_output(const InstDesc* __restrict__ d, int n) {  // t = x (+ xacc), precise precision
  const InstDesc& I = d[find_inst(d, n, blockIdx.x, true)];
  const int lb = blockIdx.x - I.eblock0, rhs = lb / I.eblk, i = (lb % I.eblk) * EW_BS + threadIdx.x;
  if (i >= I.g.V) return;
  const size_t V = (size_t)I.g.V;
  using R = ew_real<T::PA, T::PP, (T::XACC ? T::PXA : T::PA)>;
  cplx<R> v[12];
  SpinorIO<T::PA>::load(I.x, V, rhs, i, v);
  if (T::XACC) {
    cplx<R> a[12];
    SpinorIO<T::PXA>::load(I.xacc, V, rhs, i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = v[k] + a[k];
  }
  SpinorIO<T::PP>::store(I.t, V, rhs, i, v);
}

size_t fbytes(int prec, int V, int nrhs) { return (size_t)nrhs * spinor_chunks(prec) * (size_t)V * 16; }

struct ItemBufs {
  DevBuf b, t, x, r, p, q, xacc, st, partial, counter, mask;
};

template <int KIND>
struct Multi {
  using T = Traits<KIND>;
  using Rs = typename T::Rs;
  using Rp = typename T::Rp;

  static double delta() {
    char name[32];
    snprintf(name, sizeof(name), "TSM_RU_DELTA_%d", KIND);
    const char* e = getenv(name);
    return e ? atof(e) : T::DELTA;
  }

  static int solve(tsm_batch_item* items, int n, double rho, int max_iter, cudaStream_t s) {
    std::vector<ItemBufs> bufs(n);
    std::vector<InstDesc> h(n);
    int dblocks = 0, eblocks = 0, total_rhs = 0;
    for (int k = 0; k < n; ++k) {
      tsm_gauge* g = items[k].gauge;
      const int V = g->geom.V, m = items[k].nsrc;
      ItemBufs& B = bufs[k];
      TSM_TRY(B.b.reserve(fbytes(T::PP, V, m)));
      TSM_TRY(B.t.reserve(fbytes(T::PP, V, m)));
      TSM_TRY(B.x.reserve(fbytes(T::PA, V, m)));
      TSM_TRY(B.r.reserve(fbytes(T::PA, V, m)));
      TSM_TRY(B.p.reserve(fbytes(T::PS, V, m)));
      TSM_TRY(B.q.reserve(fbytes(T::PS, V, m)));
      if (T::XACC) TSM_TRY(B.xacc.reserve(fbytes(T::PXA, V, m)));
      const int nblk = (V + DSLASH_BS - 1) / DSLASH_BS;
      TSM_TRY(B.st.reserve(sizeof(RhsState) * m));
      TSM_TRY(B.partial.reserve(sizeof(double) * (size_t)nblk * m));
      TSM_TRY(B.counter.reserve(sizeof(unsigned) * m));
      TSM_CUDA(cudaMemsetAsync(B.counter.p, 0, sizeof(unsigned) * m, s));
      TSM_TRY(B.mask.reserve(sizeof(int) * m));
      InstDesc& I = h[k];
      I.g = g->geom;
      I.links_s = g->links[T::PLs].p;
      I.links_p = g->links[T::PLp].p;
      I.kappa = items[k].kappa;
      I.mup = 2.0 * items[k].kappa * items[k].mu;
      I.inv_ncomp = 1.0 / (12.0 * V);
      I.nrhs = m;
      I.nblk = nblk;
      I.dblock0 = dblocks;
      I.eblk = (V + EW_BS - 1) / EW_BS;
      I.eblock0 = eblocks;
      I.b = B.b.p;
      I.t = B.t.p;
      I.x = B.x.p;
      I.r = B.r.p;
      I.p = B.p.p;
      I.q = B.q.p;
      I.xacc = B.xacc.p;
      I.st = B.st.as<RhsState>();
      I.partial = B.partial.as<double>();
      I.counter = B.counter.as<unsigned>();
      I.mask = B.mask.as<int>();
      dblocks += nblk * m;
      eblocks += I.eblk * m;
      total_rhs += m;
      TSM_TRY(make_sources(g, items[k].noise_seed, items[k].first_src, m, T::PP, B.t.p, s));
    }
    DevBuf dd;
    TSM_TRY(dd.reserve(sizeof(InstDesc) * n));
    TSM_CUDA(cudaMemcpyAsync(dd.p, h.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice, s));
    const InstDesc* d = dd.as<InstDesc>();
    SolveParams prm;
    const double rc = cert_rho(rho, T::CERT);
    prm.rho2 = rc * rc;
    prm.delta2 = delta() * delta();
    prm.inv_ncomp = 0.0;  // per instance
    prm.max_iter = max_iter;
    prm.scaled = T::SCALED ? 1 : 0;
    count_launches(2);
    multi_dslash<Rp, +1, T::PP, T::PLp, MakeInitB<T, Rp>><<<dblocks, DSLASH_BS, 0, s>>>(d, n, MakeInitB<T, Rp>{prm});
    multi_init<T><<<eblocks, EW_BS, 0, s>>>(d, n);
    TSM_CUDA(cudaGetLastError());

    auto iteration = [&]() {
      count_launches(3);
      multi_dslash<Rs, -1, T::PS, T::PLs, MakeMp<T, Rs>><<<dblocks, DSLASH_BS, 0, s>>>(d, n, MakeMp<T, Rs>{});
      multi_dslash<Rs, +1, T::PS, T::PLs, MakeCG<T, Rs>><<<dblocks, DSLASH_BS, 0, s>>>(d, n, MakeCG<T, Rs>{prm});
      multi_pupdate<T><<<eblocks, EW_BS, 0, s>>>(d, n, 0);
    };
    const int kchunk = 8;
    cudaGraphExec_t exec = nullptr;
    {
      cudaGraph_t graph;
      TSM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      for (int it = 0; it < kchunk; ++it) iteration();
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture", __FILE__, __LINE__);
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_status(e, "cudaGraphInstantiate", __FILE__, __LINE__);
    }
    struct ExecGuard {
      cudaGraphExec_t e;
      ~ExecGuard() {
        if (e) cudaGraphExecDestroy(e);
      }
    } guard{exec};
    // counts the iterations the captured graph holds (the capture only recorded them)
    count_launches(-3LL * kchunk);

    std::vector<std::vector<RhsState>> hs(n);
    std::vector<std::vector<int>> hm(n);
    for (int k = 0; k < n; ++k) {
      hs[k].resize(items[k].nsrc);
      hm[k].resize(items[k].nsrc);
    }
    auto read_states = [&]() -> int {
      for (int k = 0; k < n; ++k)
        TSM_CUDA(cudaMemcpyAsync(hs[k].data(), bufs[k].st.p, sizeof(RhsState) * items[k].nsrc,
                                 cudaMemcpyDeviceToHost, s));
      TSM_CUDA(cudaStreamSynchronize(s));
      return TSM_OK;
    };
    const long long limit = (long long)max_iter / kchunk + 64;
    for (long long round = 0;; ++round) {
      TSM_TRY(read_states());
      bool any_ru = false;
      for (int k = 0; k < n; ++k)
        for (int r = 0; r < items[k].nsrc; ++r) {
          const RhsState& st = hs[k][r];
          const int m = (st.active && st.need_ru) || st.status == ST_ITER_CONV || st.status == ST_MAXITER;
          hm[k][r] = m;
          any_ru |= (m != 0);
        }
      if (any_ru) {
        for (int k = 0; k < n; ++k)
          TSM_CUDA(cudaMemcpyAsync(bufs[k].mask.p, hm[k].data(), sizeof(int) * items[k].nsrc, cudaMemcpyHostToDevice,
                                   s));
        count_launches(T::XACC ? 4 : 3);
        if (T::XACC) multi_fold<T><<<eblocks, EW_BS, 0, s>>>(d, n);
        multi_dslash<Rp, -1, T::PX, T::PLp, MakeRU1<T, Rp>><<<dblocks, DSLASH_BS, 0, s>>>(d, n, MakeRU1<T, Rp>{});
        multi_dslash<Rp, +1, T::PP, T::PLp, MakeRU2<T, Rp>><<<dblocks, DSLASH_BS, 0, s>>>(d, n, MakeRU2<T, Rp>{prm});
        multi_pupdate<T><<<eblocks, EW_BS, 0, s>>>(d, n, 1);
        TSM_CUDA(cudaGetLastError());
        TSM_TRY(read_states());
      }
      bool any_active = false;
      for (int k = 0; k < n; ++k)
        for (int r = 0; r < items[k].nsrc; ++r) any_active |= (hs[k][r].active != 0);
      if (!any_active) break;
      if (round > limit) return fail(TSM_ERR_CUDA, "batched solver exceeded its chunk bound");
      TSM_CUDA(cudaGraphLaunch(exec, s));
      count_launches(3LL * kchunk);
    }
    count_launches(1);
    multi_output<T><<<eblocks, EW_BS, 0, s>>>(d, n);
    TSM_CUDA(cudaGetLastError());
    int bad = 0, breakdown = 0;
    for (int k = 0; k < n; ++k) {
      tsm_gauge* g = items[k].gauge;
      TSM_TRY(spinor_convert(g, solver_output_prec(KIND), items[k].s_dev, T::PP, bufs[k].t.p, items[k].nsrc, 0, s));
      for (int r = 0; r < items[k].nsrc; ++r) {
        const RhsState& st = hs[k][r];
        const int ok = st.status == ST_DONE;
        bad += !ok;
        breakdown += st.status == ST_BREAKDOWN;
        if (items[k].stats_host) {
          tsm_solve_stats& o = items[k].stats_host[r];
          o.iterations = st.iter;
          o.reliable_updates = st.n_ru;
          o.converged = ok;
          o.restarts = st.restarts;
          o.true_residual = st.bb > 0 ? sqrt(st.true_rr / st.bb) : 0.0;
        }
      }
    }
    TSM_CUDA(cudaStreamSynchronize(s));
    if (breakdown) return fail(TSM_ERR_NONFINITE, "solver breakdown (non-finite residual)");
    if (bad) return fail(TSM_ERR_NOT_CONVERGED, "%d right-hand sides missed rho", bad);
    return TSM_OK;
  }
};

}  // namespace

int solve_batch_multi(tsm_batch_item* items, int n, int solver, double rho, int max_iter, cudaStream_t s) {
  switch (solver) {
    case TSM_SOLVER_F64: return Multi<TSM_SOLVER_F64>::solve(items, n, rho, max_iter, s);
    case TSM_SOLVER_F32_RELIABLE: return Multi<TSM_SOLVER_F32_RELIABLE>::solve(items, n, rho, max_iter, s);
    case TSM_SOLVER_LP_F16: return Multi<TSM_SOLVER_LP_F16>::solve(items, n, rho, max_iter, s);
    case TSM_SOLVER_LP_BF16: return Multi<TSM_SOLVER_LP_BF16>::solve(items, n, rho, max_iter, s);
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown solver %d", solver);
}

}  // namespace tsm
