// Backward of the one-end loops (Sec. 2.1.1) for the autograd wrapper: the
// adjoint method through Eq. 1.
//
// For a real loss l with dl/dL = G (PyTorch convention: dl/dRe L + i dl/dIm L)
// the loss is l = Re sum conj(G) L.  Writing the projected loops back on the
// sites, l = Re sum_x sum_{k,P} Omega^{k,P}(x) : F^{k,P}(x), where F are the
// open 4x4 matrices of the contraction (ultra-local D^k, derivative O^k_mu)
// and Omega^{k,P}(x) = pref_k sum_g Gamma_g w_ins(x), w_ins(x) =
// sum_n conj(G[ins, n, t]) exp(-i p_n.x).  With Theta[a][b] = g5_a Omega[a][b]:
//
//   ultra-local  l_0  = Re sum_k s^dag Theta^k chi^k
//   derivative   l_mu = Re 1/4 sum_k [ s^dag Theta^k W^k - W^0dag Theta^k chi^k ],
//                W^k = U_mu(x) chi^k(x+mu) - U_mu(x-mu)^dag chi^k(x-mu)
//
// with chi^0 = s and chi^1 = v = g5 A s.  Differentiating (Re a^dag T b:
// d/da* = T b / 2, d/db* = T^dag a / 2) gives g = dl/ds*; the W-terms are
// carried back to the sites by the transposed stencil
//   (L^dag A)(y) = U_mu(y-mu)^dag A(y-mu) - U_mu(y) A(y+mu),
// and v's share by (g5 A)^dag = g5 A.  Then, with s = M^{-1} eta,
//   lambda = M^{-dag} g,   dl/deta = 2 lambda (PyTorch convention),
//   dl/dmu = sum_r 4 kappa Im(lambda^dag g5 s) + Re(-4 i kappa Q),
// Q being the tau_3 part of l with unit prefactor (the explicit mu' in
// -2 i mu').
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dslash.cuh"
#include "internal.h"

namespace tsm {

struct GammaTable {
  int col[16][4];
  double re[16][4], im[16][4];
};

namespace {

constexpr int G_BS = 128;

__constant__ GammaTable c_gamma_grad;

// Chiral basis of include/tsm.h (same definitions as the contraction's table,
// built independently here): g_k = [[0, -i s_k], [i s_k, 0]], g_t = [[0, 1], [1, 0]].
int gamma_table(GammaTable& t) {
  double g[4][4][4][2] = {};
  const double pauli[3][2][2][2] = {
      {{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}},
      {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},
      {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}},
  };
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        const double sr = pauli[k][i][j][0], si = pauli[k][i][j][1];
        g[k][i][2 + j][0] = si;   // -i s
        g[k][i][2 + j][1] = -sr;
        g[k][2 + i][j][0] = -si;  //  i s
        g[k][2 + i][j][1] = sr;
      }
  for (int i = 0; i < 2; ++i) {
    g[3][i][2 + i][0] = 1;
    g[3][2 + i][i][0] = 1;
  }
  for (int idx = 0; idx < 16; ++idx) {
    double m[4][4][2] = {};
    for (int i = 0; i < 4; ++i) m[i][i][0] = 1;
    for (int bit = 0; bit < 4; ++bit) {
      if (!((idx >> bit) & 1)) continue;
      double r[4][4][2] = {};
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
          for (int k = 0; k < 4; ++k) {
            r[i][j][0] += m[i][k][0] * g[bit][k][j][0] - m[i][k][1] * g[bit][k][j][1];
            r[i][j][1] += m[i][k][0] * g[bit][k][j][1] + m[i][k][1] * g[bit][k][j][0];
          }
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          m[i][j][0] = r[i][j][0];
          m[i][j][1] = r[i][j][1];
        }
    }
    for (int a = 0; a < 4; ++a) {
      int nz = 0;
      for (int b = 0; b < 4; ++b)
        if (fabs(m[a][b][0]) + fabs(m[a][b][1]) > 0.5) {
          t.col[idx][a] = b;
          t.re[idx][a] = m[a][b][0];
          t.im[idx][a] = m[a][b][1];
          ++nz;
        }
      if (nz != 1) return fail(TSM_ERR_CUDA, "gamma table: row %d of Gamma_%d is not monomial", a, idx);
    }
  }
  return TSM_OK;
}

// ---------------------------------------------------------------- weights
__device__ __forceinline__ void phase(int num, int den, float& cs, float& sn) {
  sincospif(2.0f * (float)num / (float)den, &sn, &cs);
}
__device__ __forceinline__ void phase(int num, int den, double& cs, double& sn) {
  sincospi(2.0 * (double)num / (double)den, &sn, &cs);
}

// theta[f][i], f = 32 P + 16 k + 4 a + b: g5_a sum_g Gamma_g[a][b] w_ins(i), no prefactor.
template <typename R>
__global__ void __launch_bounds__(G_BS) weights_kernel(Geom geo, const double* __restrict__ grad, const int* mom,
                                                       int n_mom, const int* __restrict__ ins_active,
                                                       cplx<R>* __restrict__ theta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= geo.V) return;
  int c[4];
  site_coords(geo, i, c);
  const int lx = geo.L[0], ly = geo.L[1], lz = geo.L[2], lt = geo.L[3];
  const int n3 = lx * ly * lz;
  for (int fld = 0; fld < 10; ++fld) {  // (P, k) pairs
    const int pass = fld >> 1, k = fld & 1;
    const int ins0 = 80 * k + (pass == 0 ? 0 : 16 + 16 * (pass - 1));
    cplx<R> om[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) om[e] = mk<R>(0, 0);
    bool any = false;
    for (int gi = 0; gi < 16; ++gi) any |= (ins_active[ins0 + gi] != 0);
    if (any) {
      cplx<R> w[16];
#pragma unroll
      for (int gi = 0; gi < 16; ++gi) w[gi] = mk<R>(0, 0);
      for (int m = 0; m < n_mom; ++m) {
        // exp(-2 pi i (nx x/Lx + ny y/Ly + nz z/Lz)) from an exact integer phase
        long long ph = (long long)mom[3 * m] * c[0] * (n3 / lx) + (long long)mom[3 * m + 1] * c[1] * (n3 / ly) +
                       (long long)mom[3 * m + 2] * c[2] * (n3 / lz);
        ph %= n3;
        if (ph < 0) ph += n3;
        R cs, sn;
        phase((int)ph, n3, cs, sn);
#pragma unroll
        for (int gi = 0; gi < 16; ++gi) {
          const double* gv = grad + (((size_t)(ins0 + gi) * n_mom + m) * lt + c[3]) * 2;
          const R gr = (R)__ldg(gv), gim = (R)__ldg(gv + 1);
          // conj(G) * (cs - i sn)
          w[gi] = w[gi] + mk<R>(gr * cs - gim * sn, -gr * sn - gim * cs);
        }
      }
#pragma unroll
      for (int gi = 0; gi < 16; ++gi)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int b = c_gamma_grad.col[gi][a];
          const R gr = (R)c_gamma_grad.re[gi][a], gim = (R)c_gamma_grad.im[gi][a];
          const R sgn = a < 2 ? (R)1 : (R)-1;
          const cplx<R> v = sgn * cmul(mk<R>(gr, gim), w[gi]);
#pragma unroll
          for (int bb = 0; bb < 4; ++bb)  // the column by comparison: om stays in registers
            if (bb == b) om[4 * a + bb] = om[4 * a + bb] + v;
        }
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) theta[((size_t)(32 * pass + 16 * k + e)) * geo.V + i] = om[e];
  }
}

// (P chi)_{a c} = sum_b P[a][b] chi_{b c}
template <typename R>
__device__ __forceinline__ void mat_apply(cplx<R> (&out)[12], const cplx<R> (&p)[16], const cplx<R> (&x)[12], R scale,
                                          bool accumulate) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      cplx<R> t = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 4; ++b) cmac(t, p[4 * a + b], x[3 * b + col]);
      out[3 * a + col] = accumulate ? out[3 * a + col] + scale * t : scale * t;
    }
}
// (P^dag chi)_{a c} = sum_b conj(P[b][a]) chi_{b c}
template <typename R>
__device__ __forceinline__ void mat_apply_dag(cplx<R> (&out)[12], const cplx<R> (&p)[16], const cplx<R> (&x)[12],
                                              R scale, bool accumulate) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      cplx<R> t = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 4; ++b) cmacc(t, p[4 * b + a], x[3 * b + col]);
      out[3 * a + col] = accumulate ? out[3 * a + col] + scale * t : scale * t;
    }
}
// a^dag (P b)
template <typename R>
__device__ __forceinline__ cplx<R> form(const cplx<R> (&a)[12], const cplx<R> (&p)[16], const cplx<R> (&b)[12]) {
  cplx<R> pb[12];
  mat_apply(pb, p, b, (R)1, false);
  cplx<R> t = mk<R>(0, 0);
#pragma unroll
  for (int k = 0; k < 12; ++k) cmacc(t, a[k], pb[k]);
  return t;
}

template <typename R>
__device__ __forceinline__ void scale_mat(cplx<R> (&p)[16], cplx<R> z) {
#pragma unroll
  for (int e = 0; e < 16; ++e) p[e] = cmul(z, p[e]);
}

template <typename R>
__device__ __forceinline__ void cmatvec(cplx<R> (&w)[12], const cplx<R> (&u)[3][3], const cplx<R> (&p)[12], bool dag,
                                        R sgn) {
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> t = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (dag)
          cmacc(t, u[b][a], p[3 * sp + b]);
        else
          cmac(t, u[a][b], p[3 * sp + b]);
      }
      w[3 * sp + a] = sgn * t;
    }
}

struct LocalArgs {
  Geom g;
  const void* s;      // solutions, native
  const void* v;      // g5 A s, native
  const void* links;
  const void* theta;  // [160][V] cplx<R>
  int r;              // source index
  double mup, kappa;
  void* gs;           // out: local part of dl/ds*, native, field r
  void* gv;           // out: local part of dl/dv*, native, field r
  void* aw;           // out: [8][V] adjoint W fields (k, mu), native, single source
  double2* qpart;     // out: per-block partial of Q (tau_3 part with unit prefactor)
};

template <typename R, int PS, int PL>
__global__ void __launch_bounds__(G_BS) local_adjoint_kernel(LocalArgs a) {
  __shared__ double sh[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t V = (size_t)a.g.V;
  const cplx<R>* theta = reinterpret_cast<const cplx<R>*>(a.theta);
  cplx<R> qc = mk<R>(0, 0);
  if (i < a.g.V) {
    int c[4];
    site_coords(a.g, i, c);
    const cplx<R> pref0 = mk<R>(0, (R)(-2.0 * a.mup)), pref1 = mk<R>(2, 0);
    const cplx<R> cpref0 = conjc(pref0);
    cplx<R> s0[12], v0[12], gS[12], gV[12];
    SpinorIO<PS>::load(a.s, V, a.r, i, s0);
    SpinorIO<PS>::load(a.v, V, a.r, i, v0);
    {
      cplx<R> t0[16], t1[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        t0[e] = theta[(size_t)e * V + i];
        t1[e] = theta[(size_t)(16 + e) * V + i];
      }
      qc = form(s0, t0, s0);
      cplx<R> p0[16], p1[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        p0[e] = cmul(pref0, t0[e]);
        p1[e] = cmul(pref1, t1[e]);
      }
      mat_apply(gS, p0, s0, (R)0.5, false);
      mat_apply(gS, p1, v0, (R)0.5, true);
      mat_apply_dag(gS, p0, s0, (R)0.5, true);
      mat_apply_dag(gV, p1, s0, (R)0.5, false);
    }
    for (int mu = 0; mu < 4; ++mu) {
      const int stride = dir_stride(a.g, mu);
      const int nf = fwd_site(a.g, i, c, mu, stride), nb = bwd_site(a.g, i, c, mu, stride);
      cplx<R> uf[3][3], ub[3][3];
      LinkIO<PL>::load(a.links, V, mu, i, uf);
      LinkIO<PL>::load(a.links, V, mu, nb, ub);
      const R sf = (mu == 3 && c[3] == a.g.L[3] - 1) ? (R)a.g.bc : (R)1;
      const R sb = (mu == 3 && c[3] == 0) ? (R)a.g.bc : (R)1;
      cplx<R> t[12], w0[12], w1[12], tmp[12];
      SpinorIO<PS>::load(a.s, V, a.r, nf, t);
      cmatvec(w0, uf, t, false, sf);
      SpinorIO<PS>::load(a.s, V, a.r, nb, t);
      cmatvec(tmp, ub, t, true, sb);
#pragma unroll
      for (int k = 0; k < 12; ++k) w0[k] = w0[k] - tmp[k];
      SpinorIO<PS>::load(a.v, V, a.r, nf, t);
      cmatvec(w1, uf, t, false, sf);
      SpinorIO<PS>::load(a.v, V, a.r, nb, t);
      cmatvec(tmp, ub, t, true, sb);
#pragma unroll
      for (int k = 0; k < 12; ++k) w1[k] = w1[k] - tmp[k];
      cplx<R> t0[16], t1[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        t0[e] = theta[(size_t)(32 * (1 + mu) + e) * V + i];
        t1[e] = theta[(size_t)(32 * (1 + mu) + 16 + e) * V + i];
      }
      // unit-prefactor tau_3 part: 1/4 (s^dag T0 W0 - W0^dag T0 s)
      const cplx<R> q1 = form(s0, t0, w0), q2 = form(w0, t0, s0);
      qc = qc + (R)0.25 * (q1 - q2);
      cplx<R> p0[16], p1[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        p0[e] = cmul(pref0, t0[e]);
        p1[e] = cmul(pref1, t1[e]);
      }
      const R e8 = (R)0.125;
      mat_apply(gS, p0, w0, e8, true);
      mat_apply(gS, p1, w1, e8, true);
      mat_apply_dag(gS, p0, w0, -e8, true);
      mat_apply_dag(gV, p1, w0, -e8, true);
      cplx<R> a0[12], a1[12];
      mat_apply_dag(a0, p0, s0, e8, false);
      mat_apply(a0, p0, s0, -e8, true);
      mat_apply(a0, p1, v0, -e8, true);
      mat_apply_dag(a1, p1, s0, e8, false);
      SpinorIO<PS>::store(a.aw, V, mu, i, a0);
      SpinorIO<PS>::store(a.aw, V, 4 + mu, i, a1);
    }
    SpinorIO<PS>::store(a.gs, V, a.r, i, gS);
    SpinorIO<PS>::store(a.gv, V, a.r, i, gV);
    (void)cpref0;
  }
  double qr = block_sum((double)qc.re, sh);
  __syncthreads();
  double qi = block_sum((double)qc.im, sh);
  if (threadIdx.x == 0) a.qpart[blockIdx.x] = make_double2(qr, qi);
}

// g_s(y) += sum_mu [U(y-mu)^dag A^0_mu(y-mu) - U(y) A^0_mu(y+mu)], same for g_v with A^1.
template <typename R, int PS, int PL>
__global__ void __launch_bounds__(G_BS) transpose_stencil_kernel(Geom geo, const void* links, const void* aw, int r,
                                                                 void* gs, void* gv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= geo.V) return;
  const size_t V = (size_t)geo.V;
  int c[4];
  site_coords(geo, i, c);
  cplx<R> accs[12], accv[12];
  SpinorIO<PS>::load(gs, V, r, i, accs);
  SpinorIO<PS>::load(gv, V, r, i, accv);
  for (int mu = 0; mu < 4; ++mu) {
    const int nf = fwd_site_rt(geo, i, c, mu), nb = bwd_site_rt(geo, i, c, mu);
    cplx<R> ub[3][3], uf[3][3];
    LinkIO<PL>::load(links, V, mu, nb, ub);  // U(y - mu)
    LinkIO<PL>::load(links, V, mu, i, uf);   // U(y)
    const R sb = (mu == 3 && c[3] == 0) ? (R)geo.bc : (R)1;
    const R sf = (mu == 3 && c[3] == geo.L[3] - 1) ? (R)geo.bc : (R)1;
    cplx<R> t[12], w[12];
#pragma unroll
    for (int k = 0; k < 2; ++k) {  // unrolled: acc names one array, not a run-time choice
      cplx<R>(&acc)[12] = k == 0 ? accs : accv;
      SpinorIO<PS>::load(aw, V, 4 * k + mu, nb, t);
      cmatvec(w, ub, t, true, sb);
#pragma unroll
      for (int e = 0; e < 12; ++e) acc[e] = acc[e] + w[e];
      SpinorIO<PS>::load(aw, V, 4 * k + mu, nf, t);
      cmatvec(w, uf, t, false, sf);
#pragma unroll
      for (int e = 0; e < 12; ++e) acc[e] = acc[e] - w[e];
    }
  }
  SpinorIO<PS>::store(gs, V, r, i, accs);
  SpinorIO<PS>::store(gv, V, r, i, accv);
}

// out = a + b (fields), nrhs fields
template <int PS>
__global__ void add_fields_kernel(const void* a, const void* b, void* out, int V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= V) return;
  cplx<double> x[12], y[12];
  SpinorIO<PS>::load(a, (size_t)V, r, i, x);
  SpinorIO<PS>::load(b, (size_t)V, r, i, y);
#pragma unroll
  for (int k = 0; k < 12; ++k) x[k] = x[k] + y[k];
  SpinorIO<PS>::store(out, (size_t)V, r, i, x);
}

// per-block partials of Im(lambda^dag g5 s) for field r; out = 2 lambda (scaled copy)
template <int PS>
__global__ void __launch_bounds__(G_BS) dmu_kernel(const void* lam, const void* s, int V, double2* part, void* grad_eta,
                                                  int write_grad) {
  __shared__ double sh[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  double im = 0.0;
  if (i < V) {
    cplx<double> l[12], x[12];
    SpinorIO<PS>::load(lam, (size_t)V, r, i, l);
    SpinorIO<PS>::load(s, (size_t)V, r, i, x);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const double g5 = k < 6 ? 1.0 : -1.0;
      im += g5 * (l[k].re * x[k].im - l[k].im * x[k].re);  // Im(conj(l) x)
    }
    if (write_grad) {
#pragma unroll
      for (int k = 0; k < 12; ++k) l[k] = 2.0 * l[k];
      SpinorIO<PS>::store(grad_eta, (size_t)V, r, i, l);
    }
  }
  const double t = block_sum(im, sh);
  if (threadIdx.x == 0) part[(size_t)r * gridDim.x + blockIdx.x] = make_double2(t, 0.0);
}

}  // namespace

struct GradWorkspace {
  DevBuf theta, aw, gs, gv, tmp, lam, qpart, dpart, grad, act, mom;
  bool table = false;
};
void GradWsDeleter::operator()(GradWorkspace* w) const { delete w; }

namespace {

template <typename R, int PS>
int backward_impl(tsm_gauge* g, double kappa, double mu, const void* s_dev, int nsrc, int n_mom, const int* mom,
                  const double* grad_dev, int solver, double rho, int max_iter, double* dmu_host, void* grad_eta_dev,
                  cudaStream_t st) {
  const int V = g->geom.V, lt = g->geom.L[3];
  const size_t n_out = (size_t)160 * n_mom * lt * 2;
  std::lock_guard<std::mutex> lock(g->grad_mu);
  if (!g->grad_ws) g->grad_ws.reset(new GradWorkspace());
  GradWorkspace& w = *g->grad_ws;
  if (!w.table) {
    GammaTable t;
    TSM_TRY(gamma_table(t));
    // stream-ordered, not on the legacy default stream (see upload_gamma_table)
    TSM_CUDA(cudaMemcpyToSymbolAsync(c_gamma_grad, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st));
    TSM_CUDA(cudaStreamSynchronize(st));
    w.table = true;
  }
  // which insertions carry gradient (skipped otherwise)
  std::vector<double> gh(n_out);
  TSM_CUDA(cudaMemcpyAsync(gh.data(), grad_dev, sizeof(double) * n_out, cudaMemcpyDeviceToHost, st));
  TSM_CUDA(cudaStreamSynchronize(st));
  std::vector<int> act(160, 0);
  for (int ins = 0; ins < 160; ++ins)
    for (size_t q = 0; q < (size_t)n_mom * lt * 2; ++q) {
      const double x = gh[(size_t)ins * n_mom * lt * 2 + q];
      if (!std::isfinite(x)) return fail(TSM_ERR_NONFINITE, "non-finite loop gradient");
      if (x != 0.0) act[ins] = 1;
    }
  const size_t fb = (size_t)spinor_chunks(PS) * V * 16;
  TSM_TRY(w.theta.reserve(sizeof(cplx<R>) * 160 * (size_t)V));
  TSM_TRY(w.aw.reserve(fb * 8));
  TSM_TRY(w.gs.reserve(fb * nsrc));
  TSM_TRY(w.gv.reserve(fb * nsrc));
  TSM_TRY(w.tmp.reserve(fb * nsrc));
  TSM_TRY(w.lam.reserve(fb * nsrc));
  const int nblk = (V + G_BS - 1) / G_BS;
  TSM_TRY(w.qpart.reserve(sizeof(double2) * nblk));
  TSM_TRY(w.dpart.reserve(sizeof(double2) * (size_t)nblk * nsrc));
  TSM_TRY(w.act.reserve(sizeof(int) * 160));
  TSM_TRY(w.mom.reserve(sizeof(int) * 3 * (size_t)n_mom));
  TSM_CUDA(cudaMemcpyAsync(w.act.p, act.data(), sizeof(int) * 160, cudaMemcpyHostToDevice, st));
  TSM_CUDA(cudaMemcpyAsync(w.mom.p, mom, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, st));
  count_launches(1);
  weights_kernel<R><<<nblk, G_BS, 0, st>>>(g->geom, grad_dev, w.mom.as<int>(), n_mom, w.act.as<int>(),
                                           w.theta.as<cplx<R>>());
  TSM_CUDA(cudaGetLastError());
  // v = g5 A s into tmp
  TSM_TRY(dslash_apply_mixed(g, PS, PS, TSM_OP_A, kappa, 0.0, s_dev, w.tmp.p, nsrc, 1, st));
  double q_re = 0.0, q_im = 0.0;
  std::vector<double2> qh(nblk);
  for (int r = 0; r < nsrc; ++r) {
    LocalArgs la;
    la.g = g->geom;
    la.s = s_dev;
    la.v = w.tmp.p;
    la.links = g->links[PS].p;
    la.theta = w.theta.p;
    la.r = r;
    la.mup = 2.0 * kappa * mu;
    la.kappa = kappa;
    la.gs = w.gs.p;
    la.gv = w.gv.p;
    la.aw = w.aw.p;
    la.qpart = w.qpart.as<double2>();
    count_launches(2);
    local_adjoint_kernel<R, PS, PS><<<nblk, G_BS, 0, st>>>(la);
    transpose_stencil_kernel<R, PS, PS><<<nblk, G_BS, 0, st>>>(g->geom, g->links[PS].p, w.aw.p, r, w.gs.p, w.gv.p);
    TSM_CUDA(cudaGetLastError());
    TSM_CUDA(cudaMemcpyAsync(qh.data(), w.qpart.p, sizeof(double2) * nblk, cudaMemcpyDeviceToHost, st));
    TSM_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < nblk; ++b) {
      q_re += qh[b].x;
      q_im += qh[b].y;
    }
  }
  // g = g_s + g5 A g_v
  TSM_TRY(dslash_apply_mixed(g, PS, PS, TSM_OP_A, kappa, 0.0, w.gv.p, w.tmp.p, nsrc, 1, st));
  count_launches(1);
  add_fields_kernel<PS><<<dim3((V + 255) / 256, nsrc), 256, 0, st>>>(w.gs.p, w.tmp.p, w.gs.p, V);
  TSM_CUDA(cudaGetLastError());
  // lambda = M^{-dag} g  (M^dag x = b  <=>  M(-mu) g5 x = g5 b)
  std::vector<tsm_solve_stats> sst(nsrc);
  int rc = solve_batch_impl(g, kappa, -mu, solver, rho, max_iter, nsrc, w.gs.p, PS, 0, 0, PS, w.lam.p, 1, sst.data(),
                            st);
  if (rc != TSM_OK) return rc;
  count_launches(1);
  dmu_kernel<PS><<<dim3(nblk, nsrc), G_BS, 0, st>>>(w.lam.p, s_dev, V, w.dpart.as<double2>(), grad_eta_dev,
                                                   grad_eta_dev != nullptr);
  TSM_CUDA(cudaGetLastError());
  std::vector<double2> dh((size_t)nblk * nsrc);
  TSM_CUDA(cudaMemcpyAsync(dh.data(), w.dpart.p, sizeof(double2) * nblk * nsrc, cudaMemcpyDeviceToHost, st));
  TSM_CUDA(cudaStreamSynchronize(st));
  double im_sum = 0.0;
  for (size_t k = 0; k < dh.size(); ++k) im_sum += dh[k].x;
  // dl/dmu = 4 kappa sum Im(lambda^dag g5 s) + Re(-4 i kappa Q)
  *dmu_host = 4.0 * kappa * im_sum + 4.0 * kappa * q_im;
  (void)q_re;
  return TSM_OK;
}

}  // namespace

int loops_backward(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                   const int* mom, const double* grad_dev, int solver, double rho, int max_iter, double* dmu_host,
                   void* grad_eta_dev, cudaStream_t st) {
  if (prec == TSM_F64)
    return backward_impl<double, TSM_F64>(g, kappa, mu, s_dev, nsrc, n_mom, mom, grad_dev, solver, rho, max_iter,
                                          dmu_host, grad_eta_dev, st);
  if (prec == TSM_F32)
    return backward_impl<float, TSM_F32>(g, kappa, mu, s_dev, nsrc, n_mom, mom, grad_dev, solver, rho, max_iter,
                                         dmu_host, grad_eta_dev, st);
  return fail(TSM_ERR_INVALID_ARG, "backward takes F64 or F32 solutions");
}

}  // namespace tsm
