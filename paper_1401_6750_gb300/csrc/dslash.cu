// Stand-alone operator applications behind tsm_dslash_tm (Eq. 1's M, M^dag,
// A and M^dag M) on native fields.
#include "dslash.cuh"
#include "internal.h"

namespace tsm {

namespace {

template <typename R, int SF, int PIN, int PL, int PO>
int launch_store(const tsm_gauge* g, double kappa, double tw, const void* in, void* out, int nrhs, int gamma5,
                 cudaStream_t s) {
  DslashArgs a;
  a.g = g->geom;
  a.links = g->links[PL].p;
  a.in = in;
  a.nblk = (g->geom.V + DSLASH_BS - 1) / DSLASH_BS;
  a.nrhs = nrhs;
  a.kappa = kappa;
  a.tw = tw;
  EpiStore<R, PO> e;
  e.out = out;
  e.V = (size_t)g->geom.V;
  e.gamma5 = gamma5;
  e.red = RedSlots{nullptr, nullptr};
  count_launches(1);
  dslash_kernel<R, SF, PIN, PL, EpiStore<R, PO>><<<dslash_grid(g->geom.V, nrhs), DSLASH_BS, 0, s>>>(a, e);
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

template <int SF>
int dispatch_store(const tsm_gauge* g, int pf, int pl, double kappa, double tw, const void* in, void* out, int nrhs,
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

}  // namespace

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
      TSM_TRY(g->tmp.reserve(bytes));
      TSM_TRY(dispatch_store<-1>(g, pf, pl, kappa, mup, in, g->tmp.p, nrhs, 0, s));
      return dispatch_store<+1>(g, pf, pl, kappa, -mup, g->tmp.p, out, nrhs, gamma5, s);
    }
  }
  return fail(TSM_ERR_INVALID_ARG, "unknown operator %d", op);
}

int dslash_apply(tsm_gauge* g, int prec, int op, double kappa, double mu, const void* in, void* out, int nrhs,
                 cudaStream_t s) {
  return dslash_apply_mixed(g, prec, prec, op, kappa, mu, in, out, nrhs, 0, s);
}

}  // namespace tsm
