// Stand-alone operator applications behind tsm_dslash_tm (Eq. 1's M, M^dag,
// A and M^dag M) on native fields.
#include <stdlib.h>

#include "dslash.cuh"
#include "internal.h"

namespace tsm {

namespace {

template <typename R, int SF, int PIN, int PL, int PO>
int launch_store(tsm_gauge* g, double kappa, double tw, const void* in, void* out, int nrhs, int gamma5,
                 cudaStream_t s, int nr_forced = 0) {
  DslashArgs a;
  a.g = g->geom;
  a.links = g->links[PL].p;
  a.in = in;
  a.nblk = (g->geom.V + DSLASH_BS - 1) / DSLASH_BS;
  a.nrhs = nrhs;
  set_coeffs(a, kappa, tw);
  EpiStore<R, PO> e;
  e.out = out;
  e.V = (size_t)g->geom.V;
  e.gamma5 = gamma5;
  e.red = RedSlots{nullptr, nullptr};
  int nr = nr_forced;
  if (nr == 0) TSM_TRY(tuned_nr(g, PIN, PL, nrhs, s, &nr));
  count_launches(1);
  launch_dslash<R, SF, PIN, PL>(nr, a, e, s);
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

template <int SF>
int dispatch_store(tsm_gauge* g, int pf, int pl, double kappa, double tw, const void* in, void* out, int nrhs,
                   int gamma5, cudaStream_t s) {
  if (pf == TSM_F64 && pl == TSM_F64)
    return launch_store<double, SF, TSM_F64, TSM_F64, TSM_F64>(g, kappa, tw, in, out, nrhs, gamma5, s);
  if (pf == TSM_F32 && pl == TSM_F32)
    return launch_store<float, SF, TSM_F32, TSM_F32, TSM_F32>(g, kappa, tw, in, out, nrhs, gamma5, s);
  if (pf == TSM_F16 && pl == TSM_F16)
    return launch_store<float, SF, TSM_F16, TSM_F16, TSM_F16>(g, kappa, tw, in, out, nrhs, gamma5, s);
  if (pf == TSM_BF16 && pl == TSM_BF16)
    return launch_store<float, SF, TSM_BF16, TSM_BF16, TSM_BF16>(g, kappa, tw, in, out, nrhs, gamma5, s);
  if (pf == TSM_F32 && pl == TSM_F16)
    return launch_store<float, SF, TSM_F32, TSM_F16, TSM_F32>(g, kappa, tw, in, out, nrhs, gamma5, s);
  if (pf == TSM_F32 && pl == TSM_BF16)
    return launch_store<float, SF, TSM_F32, TSM_BF16, TSM_F32>(g, kappa, tw, in, out, nrhs, gamma5, s);
  return fail(TSM_ERR_INVALID_ARG, "no operator for field precision %d with link precision %d", pf, pl);
}

// Time the plain operator for each candidate of right-hand sides per thread.
template <typename R, int PIN, int PL>
int tune(tsm_gauge* g, int nrhs, cudaStream_t s, int* best) {
  const size_t bytes = (size_t)nrhs * spinor_chunks(PIN) * (size_t)g->geom.V * 16;
  DevBuf in, out;
  TSM_TRY(in.reserve(bytes));
  TSM_TRY(out.reserve(bytes));
  TSM_CUDA(cudaMemsetAsync(in.p, 0, bytes, s));
  EventPair ev;
  float best_t = 1e30f;
  *best = 1;
  for (int nr : {1, 2, 4}) {
    if (nr > nrhs || (sizeof(R) == 8 && nr > 2)) break;
    float tmin = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      TSM_TRY(ev.begin(s));
      TSM_TRY((launch_store<R, -1, PIN, PL, PIN>(g, 0.1, 0.01, in.p, out.p, nrhs, 0, s, nr)));
      TSM_TRY(ev.end(s));
      const float t = (float)ev.seconds();
      if (rep > 0 && t < tmin) tmin = t;
    }
    if (tmin < best_t) {
      best_t = tmin;
      *best = nr;
    }
  }
  return TSM_OK;
}

}  // namespace

int tuned_nr(tsm_gauge* g, int pin, int pl, int nrhs, cudaStream_t s, int* nr) {
  static const int forced = [] {
    const char* e = getenv("TSM_DSLASH_NR");
    return e ? atoi(e) : 0;
  }();
  if (forced == 1 || forced == 2 || forced == 4) {
    *nr = forced;
    return TSM_OK;
  }
  if (nrhs <= 1 || pin == TSM_DS) {  // float-float sums leave no registers for a second right-hand side
    *nr = 1;
    return TSM_OK;
  }
  const long long key = ((long long)pin * 8 + pl) * 100000 + nrhs;
  {
    std::lock_guard<std::mutex> l(g->tune_mu);
    auto it = g->nr_cache.find(key);
    if (it != g->nr_cache.end()) {
      *nr = it->second;
      return TSM_OK;
    }
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TSM_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) {  // cannot time inside a capture: fall back
    *nr = nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1);
    return TSM_OK;
  }
  int best = 1;
  if (pin == TSM_F64 && pl == TSM_F64) {
    TSM_TRY((tune<double, TSM_F64, TSM_F64>(g, nrhs, s, &best)));
  } else if (pin == TSM_F32 && pl == TSM_F32) {
    TSM_TRY((tune<float, TSM_F32, TSM_F32>(g, nrhs, s, &best)));
  } else if (pin == TSM_F16 && pl == TSM_F16) {
    TSM_TRY((tune<float, TSM_F16, TSM_F16>(g, nrhs, s, &best)));
  } else if (pin == TSM_BF16 && pl == TSM_BF16) {
    TSM_TRY((tune<float, TSM_BF16, TSM_BF16>(g, nrhs, s, &best)));
  } else {
    best = nrhs >= 4 ? 4 : (nrhs >= 2 ? 2 : 1);
  }
  std::lock_guard<std::mutex> l(g->tune_mu);
  g->nr_cache[key] = best;
  *nr = best;
  return TSM_OK;
}

int dslash_apply_mixed(tsm_gauge* g, int pf, int pl, int op, double kappa, double mu, const void* in, void* out,
                       int nrhs, int gamma5, cudaStream_t s) {
  if (!has_prec(g, pl)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", pl);
  const double mup = 2.0 * kappa * mu;
  switch (op) {
    case TSM_OP_M: return dispatch_store<-1>(g, pf, pl, kappa, mup, in, out, nrhs, gamma5, s);
    case TSM_OP_A: return dispatch_store<-1>(g, pf, pl, kappa, 0.0, in, out, nrhs, gamma5, s);
    case TSM_OP_MDAG: return dispatch_store<+1>(g, pf, pl, kappa, -mup, in, out, nrhs, gamma5, s);
    case TSM_OP_MDAGM: {
      const size_t bytes = (size_t)nrhs * spinor_chunks(pf) * (size_t)g->geom.V * 16;
      ScratchLease lease(g->tmp);
      TSM_TRY(lease.acquire(bytes, s));
      TSM_TRY(dispatch_store<-1>(g, pf, pl, kappa, mup, in, lease.ptr(), nrhs, 0, s));
      TSM_TRY(dispatch_store<+1>(g, pf, pl, kappa, -mup, lease.ptr(), out, nrhs, gamma5, s));
      return lease.release(s);
    }
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown operator %d", op);
}

int dslash_apply_fixed(tsm_gauge* g, int prec, int op, double kappa, double mu, const void* in, void* out, int nrhs,
                       int gamma5, int nr, cudaStream_t s) {
  if (!has_prec(g, prec)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", prec);
  const double mup = 2.0 * kappa * mu;
  if (op != TSM_OP_A && op != TSM_OP_M) return fail(TSM_ERR_INVALID_ARG, "fixed-shape launch supports M and A only");
  const double tw = (op == TSM_OP_M) ? mup : 0.0;
  switch (prec) {
    case TSM_F64: return launch_store<double, -1, TSM_F64, TSM_F64, TSM_F64>(g, kappa, tw, in, out, nrhs, gamma5, s, nr);
    case TSM_F32: return launch_store<float, -1, TSM_F32, TSM_F32, TSM_F32>(g, kappa, tw, in, out, nrhs, gamma5, s, nr);
  }
  return fail(TSM_ERR_INVALID_ARG, "fixed-shape launch supports F64 and F32 fields");
}

int hop_general(tsm_gauge* g, int prec, const void* in, const void* center, void* out, int nrhs, double c0,
                double c1, double h0, double h1, cudaStream_t s) {
  if (!has_prec(g, prec)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", prec);
  auto setup = [&](DslashArgs& a) {
    a.g = g->geom;
    a.links = g->links[prec].p;
    a.in = in;
    a.nblk = (g->geom.V + DSLASH_BS - 1) / DSLASH_BS;
    a.nrhs = nrhs;
    set_coeffs(a, 0.0, 0.0);
    set_eo(a, center, 0, c0, c1, h0, h1);
    a.general = 1;
  };
  const size_t V = (size_t)g->geom.V;
  count_launches(1);
  if (prec == TSM_F64) {
    DslashArgs a;
    setup(a);
    EpiStore<double, TSM_F64> e{out, V, 0, RedSlots{nullptr, nullptr}};
    launch_dslash<double, -1, TSM_F64, TSM_F64>(1, a, e, s);
  } else if (prec == TSM_F32) {
    DslashArgs a;
    setup(a);
    EpiStore<float, TSM_F32> e{out, V, 0, RedSlots{nullptr, nullptr}};
    launch_dslash<float, -1, TSM_F32, TSM_F32>(1, a, e, s);
  } else {
    return fail(TSM_ERR_INVALID_ARG, "general hop on F64 or F32 fields only");
  }
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

int dslash_apply(tsm_gauge* g, int prec, int op, double kappa, double mu, const void* in, void* out, int nrhs,
                 cudaStream_t s) {
  return dslash_apply_mixed(g, prec, prec, op, kappa, mu, in, out, nrhs, 0, s);
}

}  // namespace tsm
