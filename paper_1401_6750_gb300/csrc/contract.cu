// One-end-trick loops for the 160 insertions with momentum projection per
// timeslice (Sec. 2.1.1, Sec. 2.2).
//
// Following Sec. 2.2, colour is traced per site while the Dirac indices stay
// open: for phi = g5 s and chi_0 = s, chi_1 = v = g5 A s the kernel forms the
// 4x4 matrices (g_a = diag(g5)_a)
//
//   ultra-local  D^k[a][b]   = g_a sum_c conj(s_ac) chi^k_bc
//   derivative   O^k_mu[a][b] = 1/4 g_a sum_c [ conj(s_ac) W^k_bc - conj(W^0_ac) chi^k_bc ]
//                W^k = U_mu(x) chi^k(x+mu) - U_mu(x-mu)^dag chi^k(x-mu)
//
// (the four terms of the symmetric covariant insertion collapse into two
// outer products because U commutes with g5), summed over the sources of
// the batch.  Each Gamma insertion is formed from the 4x4 matrix at the site
// ("by transposition and multiplication", Sec. 2.2):
//   T_g = sum_ab Gamma_g[a][b] D[a][b],
// a monomial matrix in the chiral basis, so 4 terms per insertion, giving
// 10 x 16 = 160 complex fields per site.  (Forming the insertions after the
// projection instead, as the paper's double-precision code could, makes the
// FP32 sums over sites carry the large diagonal entries of D whose
// combination cancels -- g5 has +1 and -1 on the diagonal -- and costs the
// FP32 contraction a decade of relative accuracy on those insertions.)
// These fields are projected to momenta with a separable transform, x then y
// inside a (z, t)-plane block (FP32, short sums), and z in FP64 by a second
// kernel, which also applies the derivative shift and the flavour
// prefactors, pref_0 = -2 i mu', pref_1 = 2.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <utility>
#include <vector>

#include "dslash.cuh"
#include "internal.h"

namespace tsm {

// ---------------------------------------------------------------- Gamma table
struct GammaTable {
  int col[16][4];      // Gamma_g[a][col] is the only non-zero of row a
  double re[16][4], im[16][4];
};
__constant__ GammaTable c_gamma;

// The same insertion matrices as compile-time monomials: Gamma_g has one
// non-zero per row a, the power i^ph[a] at column col[a].  The site-field
// kernels form the insertion traces with them per site (before any sum over
// sites), so that no FP32 sum ever combines the large, nearly cancelling
// diagonal entries of the open Dirac matrices; the host table above is
// checked against these at upload.
struct Mono4 {
  int col[4];
  int ph[4];
};
constexpr Mono4 mono_mul(const Mono4& a, const Mono4& b) {
  Mono4 c{};
  for (int r = 0; r < 4; ++r) {
    c.col[r] = b.col[a.col[r]];
    c.ph[r] = (a.ph[r] + b.ph[a.col[r]]) & 3;
  }
  return c;
}
// chiral basis of include/tsm.h, read off row by row:
//   g_x: (0,3) -i, (1,2) -i, (2,1) i, (3,0) i     g_y: (0,3) -1, (1,2) 1, (2,1) 1, (3,0) -1
//   g_z: (0,2) -i, (1,3) i, (2,0) i, (3,1) -i     g_t: (0,2) 1, (1,3) 1, (2,0) 1, (3,1) 1
constexpr Mono4 gamma_base(int mu) {
  return mu == 0   ? Mono4{{3, 2, 1, 0}, {3, 3, 1, 1}}
         : mu == 1 ? Mono4{{3, 2, 1, 0}, {2, 0, 0, 2}}
         : mu == 2 ? Mono4{{2, 3, 0, 1}, {3, 1, 1, 3}}
                   : Mono4{{2, 3, 0, 1}, {0, 0, 0, 0}};
}
// Gamma_g = g_x^{b0} g_y^{b1} g_z^{b2} g_t^{b3}
constexpr Mono4 gamma_ins(int g) {
  Mono4 m{{0, 1, 2, 3}, {0, 0, 0, 0}};
  for (int bit = 0; bit < 4; ++bit)
    if ((g >> bit) & 1) m = mono_mul(m, gamma_base(bit));
  return m;
}

template <int PH, typename R>
__device__ __forceinline__ cplx<R> times_ipow(cplx<R> z) {
  return PH == 0 ? z : (PH == 1 ? mk<R>(-z.im, z.re) : (PH == 2 ? mk<R>(-z.re, -z.im) : mk<R>(z.im, -z.re)));
}
// sum_a Gamma_g[a][col_a] rowfac(a) m[a][col_a], rowfac = +scale for a < 2 (the g5 of phi = g5 s), -scale else
template <int G, typename R>
__device__ __forceinline__ cplx<R> insertion_trace(const cplx<R> (&m)[16], R scale) {
  constexpr Mono4 q = gamma_ins(G);
  cplx<R> t = scale * times_ipow<q.ph[0]>(m[0 * 4 + q.col[0]]);
  t = t + scale * times_ipow<q.ph[1]>(m[1 * 4 + q.col[1]]);
  t = t - scale * times_ipow<q.ph[2]>(m[2 * 4 + q.col[2]]);
  t = t - scale * times_ipow<q.ph[3]>(m[3 * 4 + q.col[3]]);
  return t;
}
template <typename R, int... G>
__device__ __forceinline__ void store_traces(cplx<R>* out, size_t V, const cplx<R> (&m)[16], R scale,
                                             std::integer_sequence<int, G...>) {
  ((out[(size_t)G * V] = insertion_trace<G>(m, scale)), ...);
}

// The standard estimator's two traces of a 4x4 matrix m (no g5 row factor):
//   u:  sum_a Gamma_g[a][b] m[a][b]
//   d:  sum_a g5_a g5_b conj(Gamma_g[a][b]) m[b][a]   (b = col_a),
// the second being the trace with g5 Gamma_g^dag g5 that the d flavour
// needs (its projection is taken at -p and conjugated afterwards).
template <int G, typename R>
__device__ __forceinline__ void std_traces(cplx<R>& tu, cplx<R>& td, const cplx<R> (&m)[16], R scale) {
  constexpr Mono4 q = gamma_ins(G);
  tu = mk<R>(0, 0);
  td = mk<R>(0, 0);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int b = q.col[a], ph = q.ph[a];
    const cplx<R> x = m[4 * a + b], y = m[4 * b + a];
    // u: i^ph x;  d: sg conj(i^ph) y = sg i^(-ph) y
    const cplx<R> ux = ph == 0 ? x : (ph == 1 ? mk<R>(-x.im, x.re) : (ph == 2 ? mk<R>(-x.re, -x.im) : mk<R>(x.im, -x.re)));
    const cplx<R> dy = ph == 0 ? y : (ph == 1 ? mk<R>(y.im, -y.re) : (ph == 2 ? mk<R>(-y.re, -y.im) : mk<R>(-y.im, y.re)));
    const R sg = ((a < 2) == (b < 2)) ? scale : -scale;
    tu = tu + scale * ux;
    td = td + sg * dy;
  }
}
// The two flavour combinations per site: d = sd conj(t_d) (sd = +1 for the
// ultra-local pass, -1 for the derivative ones: the d form of the
// derivative's two terms comes with the opposite sign), out[g] = u - d
// (with tau_3), out[16 + g] = u + d.  The conjugate is taken per site, so
// that no sum over sites ever carries the nearly equal real parts of u and d.
template <int G, typename R>
__device__ __forceinline__ void store_std_combos(cplx<R>* out, size_t V, const cplx<R> (&m)[16], R scale, R sd) {
  cplx<R> tu, td;
  std_traces<G>(tu, td, m, scale);
  const cplx<R> d = mk<R>(sd * td.re, -sd * td.im);
  out[(size_t)G * V] = tu - d;
  out[(size_t)(16 + G) * V] = tu + d;
}
template <typename R, int... G>
__device__ __forceinline__ void store_std_traces(cplx<R>* out, size_t V, const cplx<R> (&m)[16], R scale, R sd,
                                                 std::integer_sequence<int, G...>) {
  (store_std_combos<G>(out, V, m, scale, sd), ...);
}

namespace {

struct HostCplx {
  double re, im;
};
typedef HostCplx Mat4[4][4];

void mat_mul(const Mat4 a, const Mat4 b, Mat4 out) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double re = 0, im = 0;
      for (int k = 0; k < 4; ++k) {
        re += a[i][k].re * b[k][j].re - a[i][k].im * b[k][j].im;
        im += a[i][k].re * b[k][j].im + a[i][k].im * b[k][j].re;
      }
      out[i][j] = HostCplx{re, im};
    }
}

// Chiral basis of include/tsm.h: g_k = [[0, -i s_k], [i s_k, 0]], g_t = [[0, 1], [1, 0]].
void chiral_gammas(Mat4 g[4]) {
  const HostCplx pauli[3][2][2] = {
      {{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}},
      {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},
      {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}},
  };
  for (int m = 0; m < 4; ++m)
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) g[m][i][j] = HostCplx{0, 0};
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        const HostCplx s = pauli[k][i][j];
        g[k][i][2 + j] = HostCplx{s.im, -s.re};   // -i s
        g[k][2 + i][j] = HostCplx{-s.im, s.re};   //  i s
      }
  for (int i = 0; i < 2; ++i) {
    g[3][i][2 + i] = HostCplx{1, 0};
    g[3][2 + i][i] = HostCplx{1, 0};
  }
}

int build_gamma_table(GammaTable& t) {
  Mat4 g[4];
  chiral_gammas(g);
  for (int idx = 0; idx < 16; ++idx) {
    Mat4 m, tmp;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) m[i][j] = HostCplx{i == j ? 1.0 : 0.0, 0.0};
    for (int bit = 0; bit < 4; ++bit)
      if ((idx >> bit) & 1) {
        mat_mul(m, g[bit], tmp);
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) m[i][j] = tmp[i][j];
      }
    for (int a = 0; a < 4; ++a) {
      int nz = 0;
      for (int b = 0; b < 4; ++b)
        if (fabs(m[a][b].re) + fabs(m[a][b].im) > 0.5) {
          t.col[idx][a] = b;
          t.re[idx][a] = m[a][b].re;
          t.im[idx][a] = m[a][b].im;
          ++nz;
        }
      if (nz != 1) return fail(TSM_ERR_CUDA, "gamma table: Gamma_%d row %d is not monomial", idx, a);
    }
  }
  return TSM_OK;
}

// Build the table and copy it to c_gamma on stream st, waiting for the copy:
// the copy is ordered on the caller's stream rather than on the legacy
// default stream, which would synchronise implicitly with (and so
// invalidate) a graph capture on a blocking stream of another host thread.
int upload_gamma_table(cudaStream_t st) {
  GammaTable t;  // lives until the copy has completed (synchronised below)
  TSM_TRY(build_gamma_table(t));
  for (int g = 0; g < 16; ++g) {
    const Mono4 q = gamma_ins(g);
    for (int a = 0; a < 4; ++a) {
      const double pr[4] = {1, 0, -1, 0}, pi[4] = {0, 1, 0, -1};
      if (t.col[g][a] != q.col[a] || t.re[g][a] != pr[q.ph[a]] || t.im[g][a] != pi[q.ph[a]])
        return fail(TSM_ERR_CUDA, "insertion table mismatch at Gamma_%d row %d", g, a);
    }
  }
  TSM_CUDA(cudaMemcpyToSymbolAsync(c_gamma, &t, sizeof(t), 0, cudaMemcpyHostToDevice, st));
  TSM_CUDA(cudaStreamSynchronize(st));
  return TSM_OK;
}

constexpr int NF = 32;       // fields per pass: 2 flavour structures x 16
constexpr int FLD_BS = 128;  // site-field kernel block
constexpr int XY_BS = 256;   // x/y transform block
constexpr int XY_NC = 7;     // momenta per accumulator set
constexpr int Z_BS = 256;
// grid of project_z_kernel: (timeslice, 10 field groups, slices of Z_BS (momentum, field) pairs)
inline dim3 z_grid(int lt, int n_mom) {
  return dim3(lt, 10, (unsigned)std::min((n_mom * 16 + Z_BS - 1) / Z_BS, 65535));
}

// Site fields (summed over the sources) in F[(pass*NF + f) * V + i], site fastest.
template <typename R>
struct FieldArgs {
  Geom g;
  const void* s;
  const void* v;
  const void* links;
  int nsrc;
  cplx<R>* F;
};

template <typename R>
__device__ __forceinline__ void matvec(cplx<R> (&w)[12], const cplx<R> (&u)[3][3], const cplx<R> (&p)[12], R sgn) {
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> t = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; ++b) cmac(t, u[a][b], p[3 * sp + b]);
      w[3 * sp + a] = sgn * t;
    }
}

// acc[a*4+b] += sum_c conj(l_ac) r_bc   (times -1 when SUB)
template <bool SUB, typename R>
__device__ __forceinline__ void outer(cplx<R> (&acc)[16], const cplx<R> (&l)[12], const cplx<R> (&r)[12]) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (SUB)
          cmacc(acc[4 * a + b], mk<R>(-l[3 * a + c].re, -l[3 * a + c].im), r[3 * b + c]);
        else
          cmacc(acc[4 * a + b], l[3 * a + c], r[3 * b + c]);
      }
}

// The symmetric covariant derivative at x collapses onto forward products:
//   O_mu(x) = 1/4 [D_mu(x) + D_mu(x - mu)],
//   D^0_mu(y)[a][b] = g_a (M[a][b] - conj(M[b][a])),  M = sum_c conj(s_ac(y)) (U_mu(y) s(y+mu))_bc
//   D^1_mu(y)[a][b] = g_a sum_c [conj(s_ac(y)) (U_mu(y) v(y+mu))_bc - conj((U_mu(y) s(y+mu))_ac) v_bc(y)]
// (the two backward terms of O at x are the forward products rooted at
// x - mu).  The shift is applied after the projection: a phase
// (1 + e^{-i p_mu}) for spatial mu, the sum of timeslices t and t-1 for mu = t.
// Pass 0 holds the ultra-local D^0 = g_a sum_c conj(s_ac) s_bc and D^1 with v.
template <typename R, int PS, int PL>
__global__ void __launch_bounds__(FLD_BS, sizeof(R) == 4 ? 3 : 1) contract_fields_kernel(FieldArgs<R> a) {
  const int pass = blockIdx.x % 5;
  const int i = (blockIdx.x / 5) * FLD_BS + threadIdx.x;
  if (i >= a.g.V) return;
  const size_t V = (size_t)a.g.V;
  cplx<R> m0[16], m1[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) m0[k] = m1[k] = mk<R>(0, 0);
  R scale = (R)1;
  if (pass == 0) {
    for (int r = 0; r < a.nsrc; ++r) {
      cplx<R> s0[12], v0[12];
      SpinorIO<PS>::load(a.s, V, r, i, s0);
      SpinorIO<PS>::load(a.v, V, r, i, v0);
      outer<false>(m0, s0, s0);
      outer<false>(m1, s0, v0);
    }
  } else {
    const int mu = pass - 1;
    int c[4];
    site_coords(a.g, i, c);
    const int nf = fwd_site_rt(a.g, i, c, mu);
    cplx<R> u[3][3];
    LinkIO<PL>::load(a.links, V, mu, i, u);
    const R sf = (mu == 3 && c[3] == a.g.L[3] - 1) ? (R)a.g.bc : (R)1;
    for (int r = 0; r < a.nsrc; ++r) {
      cplx<R> t[12], w[12], s0[12];
      SpinorIO<PS>::load(a.s, V, r, nf, t);
      matvec(w, u, t, sf);                   // U s(y+mu)
      SpinorIO<PS>::load(a.s, V, r, i, s0);
      outer<false>(m0, s0, w);
      SpinorIO<PS>::load(a.v, V, r, i, t);
      outer<true>(m1, w, t);                 // - conj(U s(y+mu)) v(y)
      SpinorIO<PS>::load(a.v, V, r, nf, t);
      matvec(w, u, t, sf);                   // U v(y+mu)
      outer<false>(m1, s0, w);
    }
    // D^0 = M - M^dag (before the g_a row factor)
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p; q < 4; ++q) {
        const cplx<R> x = m0[4 * p + q], y = m0[4 * q + p];
        m0[4 * p + q] = mk<R>(x.re - y.re, x.im + y.im);
        m0[4 * q + p] = mk<R>(y.re - x.re, y.im + x.im);
      }
    scale = (R)0.25;
  }
  cplx<R>* out = a.F + (size_t)pass * NF * V + i;
  store_traces(out, V, m0, scale, std::make_integer_sequence<int, 16>{});
  store_traces(out + 16 * V, V, m1, scale, std::make_integer_sequence<int, 16>{});
}

// The same site fields with FP32 sums in packed pairs (two-wide FP32 FMA):
// a spinor is held as pairs over adjacent spins, re[c][h] = (x[6h + c].re,
// x[6h + 3 + c].re) for spins (2h, 2h + 1), and a 4x4 Dirac matrix as pairs
// over adjacent columns, re[a][h] = (m[a][2h].re, m[a][2h + 1].re).
struct SpinP {
  float2 re[3][2], im[3][2];
};
struct Mat4P {
  float2 re[4][2], im[4][2];
};

__device__ __forceinline__ float2 bc2f(float v) { return make_float2(v, v); }

__device__ __forceinline__ void pack_spin(SpinP& p, const cplx<float> (&x)[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      p.re[c][h] = make_float2(x[6 * h + c].re, x[6 * h + 3 + c].re);
      p.im[c][h] = make_float2(x[6 * h + c].im, x[6 * h + 3 + c].im);
    }
}
// component (spin a, colour c) of either form
__device__ __forceinline__ cplx<float> comp(const cplx<float> (&x)[12], int a, int c) { return x[3 * a + c]; }
__device__ __forceinline__ cplx<float> comp(const SpinP& x, int a, int c) {
  const float2 r = x.re[c][a >> 1], i = x.im[c][a >> 1];
  return (a & 1) ? mk<float>(r.y, i.y) : mk<float>(r.x, i.x);
}

// w = U p for all four spins (pairs over spins)
__device__ __forceinline__ void matvec_p(SpinP& w, const cplx<float> (&u)[3][3], const SpinP& p) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float2 wr = __fmul2_rn(bc2f(u[a][0].re), p.re[0][h]);
      float2 wi = __fmul2_rn(bc2f(u[a][0].re), p.im[0][h]);
      wr = __ffma2_rn(bc2f(-u[a][0].im), p.im[0][h], wr);
      wi = __ffma2_rn(bc2f(u[a][0].im), p.re[0][h], wi);
#pragma unroll
      for (int b = 1; b < 3; ++b) {
        wr = __ffma2_rn(bc2f(u[a][b].re), p.re[b][h], wr);
        wr = __ffma2_rn(bc2f(-u[a][b].im), p.im[b][h], wr);
        wi = __ffma2_rn(bc2f(u[a][b].re), p.im[b][h], wi);
        wi = __ffma2_rn(bc2f(u[a][b].im), p.re[b][h], wi);
      }
      w.re[a][h] = wr;
      w.im[a][h] = wi;
    }
}

// m[a][b] += sum_c conj(l_ac) r_bc   (times -1 when SUB); r in pairs over spins b
template <bool SUB, class L>
__device__ __forceinline__ void outer_p(Mat4P& m, const L& l, const SpinP& r) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cplx<float> x = comp(l, a, c);
      const float lr = SUB ? -x.re : x.re, li = SUB ? -x.im : x.im;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        m.re[a][h] = __ffma2_rn(bc2f(lr), r.re[c][h], m.re[a][h]);
        m.re[a][h] = __ffma2_rn(bc2f(li), r.im[c][h], m.re[a][h]);
        m.im[a][h] = __ffma2_rn(bc2f(lr), r.im[c][h], m.im[a][h]);
        m.im[a][h] = __ffma2_rn(bc2f(-li), r.re[c][h], m.im[a][h]);
      }
    }
}

__device__ __forceinline__ void unpack_mat(cplx<float> (&m)[16], const Mat4P& p) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      m[4 * a + 2 * h] = mk<float>(p.re[a][h].x, p.im[a][h].x);
      m[4 * a + 2 * h + 1] = mk<float>(p.re[a][h].y, p.im[a][h].y);
    }
}

template <int PS, int PL>
__global__ void __launch_bounds__(FLD_BS, 3) contract_fields_pairs_kernel(FieldArgs<float> a) {
  const int pass = blockIdx.x % 5;
  const int i = (blockIdx.x / 5) * FLD_BS + threadIdx.x;
  if (i >= a.g.V) return;
  const size_t V = (size_t)a.g.V;
  Mat4P p0, p1;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int h = 0; h < 2; ++h) p0.re[x][h] = p0.im[x][h] = p1.re[x][h] = p1.im[x][h] = make_float2(0.0f, 0.0f);
  float scale = 1.0f;
  if (pass == 0) {
    for (int r = 0; r < a.nsrc; ++r) {
      cplx<float> s0[12], v0[12];
      SpinorIO<PS>::load(a.s, V, r, i, s0);
      SpinorIO<PS>::load(a.v, V, r, i, v0);
      SpinP sp, vp;
      pack_spin(sp, s0);
      pack_spin(vp, v0);
      outer_p<false>(p0, s0, sp);
      outer_p<false>(p1, s0, vp);
    }
  } else {
    const int mu = pass - 1;
    int c[4];
    site_coords(a.g, i, c);
    const int nf = fwd_site_rt(a.g, i, c, mu);
    cplx<float> u[3][3];
    LinkIO<PL>::load(a.links, V, mu, i, u);
    if (mu == 3 && c[3] == a.g.L[3] - 1 && a.g.bc < 0) {  // boundary sign folded into the link
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) u[x][y] = mk<float>(-u[x][y].re, -u[x][y].im);
    }
    for (int r = 0; r < a.nsrc; ++r) {
      cplx<float> t[12], s0[12];
      SpinP tp, w;
      SpinorIO<PS>::load(a.s, V, r, nf, t);
      pack_spin(tp, t);
      matvec_p(w, u, tp);                  // U s(y+mu)
      SpinorIO<PS>::load(a.s, V, r, i, s0);
      outer_p<false>(p0, s0, w);
      SpinorIO<PS>::load(a.v, V, r, i, t);
      pack_spin(tp, t);
      outer_p<true>(p1, w, tp);            // - conj(U s(y+mu)) v(y)
      SpinorIO<PS>::load(a.v, V, r, nf, t);
      pack_spin(tp, t);
      matvec_p(w, u, tp);                  // U v(y+mu)
      outer_p<false>(p1, s0, w);
    }
    scale = 0.25f;
  }
  cplx<float> m0[16], m1[16];
  unpack_mat(m0, p0);
  unpack_mat(m1, p1);
  if (pass != 0) {  // D^0 = M - M^dag (before the g_a row factor)
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p; q < 4; ++q) {
        const cplx<float> x = m0[4 * p + q], y = m0[4 * q + p];
        m0[4 * p + q] = mk<float>(x.re - y.re, x.im + y.im);
        m0[4 * q + p] = mk<float>(y.re - x.re, y.im + x.im);
      }
  }
  cplx<float>* out = a.F + (size_t)pass * NF * V + i;
  store_traces(out, V, m0, scale, std::make_integer_sequence<int, 16>{});
  store_traces(out + 16 * V, V, m1, scale, std::make_integer_sequence<int, 16>{});
}

// Partial sums of the x/y transform per field precision: the FP32 sums are
// stored as they are (float2; the float-float z sum takes them exactly),
// the FP64 ones as double2.
template <typename R>
struct PartOf {
  using type = double2;
};
template <>
struct PartOf<float> {
  using type = float2;
};

// Twiddle tables of the x/y transform hold e^{-2 pi i m / L} in the field precision.
template <typename R>
struct TwOf {
  using type = cplx<R>;
};

__device__ __forceinline__ void twiddle(cplx<float>& o, int m, int L) {
  float sn, cs;
  sincospif(2.0f * (float)m / (float)L, &sn, &cs);
  o = mk<float>(cs, -sn);
}
__device__ __forceinline__ void twiddle(cplx<double>& o, int m, int L) {
  double sn, cs;
  sincospi(2.0 * (double)m / (double)L, &sn, &cs);
  o = mk<double>(cs, -sn);
}

__device__ __forceinline__ void store_part(float2* p, cplx<float> v) { *p = make_float2(v.re, v.im); }
__device__ __forceinline__ void store_part(double2* p, cplx<double> v) { *p = make_double2(v.re, v.im); }

// x then y transform of the site fields on one (z, t) plane:
//   part[plane][(n_x, n_y)][f] = sum_{x,y} F_f(x, y) e^{-2 pi i (n_x x / Lx + n_y y / Ly)}
// Block (plane, chunk of nfc fields).  The chunk's planes (Lx Ly contiguous
// values per field) are first copied to shared memory with coalesced loads,
// rows padded to Lx + 1 values so that the row-wise reads below spread over
// the banks; x: one thread per (field, row) keeps XY_NC momenta in flight;
// y: one thread per (field, n_x) over the rows; the chunk's results are
// staged so that the stores run along f.
template <typename R>
__global__ void __launch_bounds__(XY_BS, 4) contract_xy_kernel(const cplx<R>* __restrict__ F, Geom g, int rad,
                                                            int nfc, int nfields,
                                                            typename PartOf<R>::type* __restrict__ part) {
  using TW = typename TwOf<R>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lx = g.L[0], ly = g.L[1], lxp = lx + 1;
  const int nx = 2 * rad + 1, nxy = nx * nx;
  const int nchunk = nfields / nfc;
  const int plane = blockIdx.x / nchunk;  // z + Lz * t
  const int f0 = (blockIdx.x % nchunk) * nfc;
  cplx<R>* S = reinterpret_cast<cplx<R>*>(smem_raw);  // [nfc][ly][lx + 1]
  cplx<R>* X = S + (size_t)nfc * ly * lxp;             // [nfc][ly][nx]
  cplx<R>* Y = X + (size_t)nfc * ly * nx;              // [nxy][nfc]
  const size_t tw_off = ((size_t)(Y + (size_t)nxy * nfc - S) * sizeof(cplx<R>) + 15) & ~(size_t)15;
  TW* twx = reinterpret_cast<TW*>(smem_raw + tw_off);  // [lx][nx], 16-byte aligned
  TW* twy = twx + (size_t)lx * nx;                     // [ly][nx]
  const size_t V = (size_t)g.V;
  const int pv = lx * ly;
  const cplx<R>* Fp = F + (size_t)f0 * V + (size_t)plane * pv;
  // plane index q -> padded row offset, split once per thread and reused for every field of the chunk
  for (int q = threadIdx.x; q < pv; q += blockDim.x) {
    const int row = q / lx;
    cplx<R>* dst = S + row * lxp + (q - row * lx);
    const cplx<R>* src = Fp + q;
    for (int f = 0; f < nfc; ++f) dst[(size_t)f * ly * lxp] = src[(size_t)f * V];
  }
  for (int k = threadIdx.x; k < nx * lx; k += blockDim.x) {
    const int x = k / nx, n = k % nx - rad;
    twiddle(twx[k], ((n * x) % lx + lx) % lx, lx);
  }
  for (int k = threadIdx.x; k < nx * ly; k += blockDim.x) {
    const int y = k / nx, n = k % nx - rad;
    twiddle(twy[k], ((n * y) % ly + ly) % ly, ly);
  }
  __syncthreads();
  for (int task = threadIdx.x; task < nfc * ly; task += blockDim.x) {
    const int row = task % ly, f = task / ly;
    const cplx<R>* src = S + ((size_t)f * ly + row) * lxp;
    cplx<R>* dst = X + ((size_t)f * ly + row) * nx;
    for (int n0 = 0; n0 < nx; n0 += XY_NC) {
      cplx<R> acc[XY_NC];
#pragma unroll
      for (int j = 0; j < XY_NC; ++j) acc[j] = mk<R>(0, 0);
#pragma unroll 6
      for (int x = 0; x < lx; ++x) {
        const cplx<R> v = src[x];
        const TW* tw = twx + (size_t)x * nx + n0;
#pragma unroll
        for (int j = 0; j < XY_NC; ++j)
          if (n0 + j < nx) cmac(acc[j], v, tw[j]);
      }
#pragma unroll
      for (int j = 0; j < XY_NC; ++j)
        if (n0 + j < nx) dst[n0 + j] = acc[j];
    }
  }
  __syncthreads();
  for (int task = threadIdx.x; task < nfc * nx; task += blockDim.x) {
    const int f = task % nfc, n_x = task / nfc;
    const cplx<R>* src = X + (size_t)f * ly * nx + n_x;
    for (int n0 = 0; n0 < nx; n0 += XY_NC) {
      cplx<R> acc[XY_NC];
#pragma unroll
      for (int j = 0; j < XY_NC; ++j) acc[j] = mk<R>(0, 0);
#pragma unroll 6
      for (int row = 0; row < ly; ++row) {
        const cplx<R> v = src[(size_t)row * nx];
        const TW* tw = twy + (size_t)row * nx + n0;
#pragma unroll
        for (int j = 0; j < XY_NC; ++j)
          if (n0 + j < nx) cmac(acc[j], v, tw[j]);
      }
#pragma unroll
      for (int j = 0; j < XY_NC; ++j)
        if (n0 + j < nx) Y[((size_t)n_x * nx + n0 + j) * nfc + f] = acc[j];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nxy * nfc; k += blockDim.x) {
    const int f = k % nfc, nn = k / nfc;
    store_part(part + ((size_t)plane * nxy + nn) * nfields + f0 + f, Y[k]);
  }
}

// Arithmetic of the z sum per part type: FP64 for FP64 partial sums,
// float-float (about 44 bits, on the FP32 pipes) for FP32 ones, which it
// takes exactly.  GB300's FP64 pipe is 1/64 of FP32: in FP64 this sum kept
// it 87% busy.
template <typename PT>
struct ZReal {
  using type = double;
};
template <>
struct ZReal<float2> {
  using type = dsf;
};
template <typename Z>
__device__ __forceinline__ cplx<Z> zload(const float2& p) {
  return mk<Z>(Z(p.x), Z(p.y));
}
template <typename Z>
__device__ __forceinline__ cplx<Z> zload(const double2& p) {
  return mk<Z>(Z(p.x), Z(p.y));
}
__device__ __forceinline__ double zdouble(double v) { return v; }
__device__ __forceinline__ double zdouble(dsf v) { return (double)v; }

// z transform, the derivative shift and the loop prefactor.  Block (t,
// group, slice): group = 2 pass + k holds 16 fields of one pass; slice z
// takes the (momentum, field) pairs z * Z_BS .. z * Z_BS + Z_BS - 1, one per
// thread, written directly.  The block's phases (z twiddles, and the shift
// factors of its direction) are tabulated in shared memory first.
template <typename PT>
__global__ void __launch_bounds__(Z_BS) project_z_kernel(const PT* __restrict__ part, const int* __restrict__ mom,
                                                         int n_mom, Geom g, int rad, double mup, double* out,
                                                         int accumulate, int unit_prefactor) {
  using Z = typename ZReal<PT>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lz = g.L[2], lt = g.L[3];
  const int t = blockIdx.x, group = blockIdx.y;
  const int pass = group >> 1, k = group & 1;
  const int nx = 2 * rad + 1, nxy = nx * nx;
  cplx<Z>* twz = reinterpret_cast<cplx<Z>*>(smem_raw);  // [nx][lz]: e^{-2 pi i n z / Lz}
  cplx<Z>* shf = twz + (size_t)nx * lz;                   // [nx]: 1 + e^{-2 pi i n / L_mu}, mu = pass - 1
  cplx<Z>* root = shf + nx;                               // [lz]: e^{-2 pi i m / Lz}
  for (int q = threadIdx.x; q < lz + nx; q += blockDim.x) {  // the Lz + nx distinct phases, in FP64
    double sn, cs;
    if (q < lz) {
      sincospi(2.0 * (double)q / (double)lz, &sn, &cs);
      root[q] = mk<Z>(Z(cs), Z(-sn));
    } else if (pass >= 1 && pass <= 3) {
      const int n = q - lz - rad, L = g.L[pass - 1];
      sincospi(2.0 * (double)(((n % L) + L) % L) / (double)L, &sn, &cs);
      shf[n + rad] = mk<Z>(Z(1.0 + cs), Z(-sn));
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < nx * lz; q += blockDim.x) {
    const int n = q / lz - rad, zz = q % lz;
    twz[q] = root[((n * zz) % lz + lz) % lz];
  }
  __syncthreads();
  const int field0 = pass * NF + k * 16;
  const int tm1 = (t + lt - 1) % lt;
  // prefactor: k = 0 -> -2 i mu', k = 1 -> 2 (the fields are the insertion traces already);
  // 1 for both when the fields carry their flavour factors (standard estimator)
  const double pre = unit_prefactor ? 1.0 : ((k == 0) ? 0.0 : 2.0);
  const double pim = (unit_prefactor || k != 0) ? 0.0 : -2.0 * mup;
  for (int q = blockIdx.z * blockDim.x + threadIdx.x; q < n_mom * 16; q += gridDim.z * blockDim.x) {
    const int m = q / 16, e = q % 16;
    const int mx = mom[3 * m], my = mom[3 * m + 1], mz = mom[3 * m + 2];
    const int nn = (mx + rad) * nx + (my + rad);
    const cplx<Z>* tw = twz + (size_t)(mz + rad) * lz;
    cplx<Z> acc = mk<Z>(Z(0.0), Z(0.0));
    for (int zz = 0; zz < lz; ++zz) {
      cplx<Z> p = zload<Z>(part[((size_t)(zz + lz * t) * nxy + nn) * 160 + field0 + e]);
      if (pass == 4)  // O_t(t) = D_t(t) + D_t(t - 1)
        p = p + zload<Z>(part[((size_t)(zz + lz * tm1) * nxy + nn) * 160 + field0 + e]);
      acc = acc + cmul(p, tw[zz]);
    }
    if (pass >= 1 && pass <= 3)  // O_mu(p) = (1 + e^{-2 pi i n_mu / L_mu}) D_mu(p)
      acc = cmul(acc, shf[(pass == 1 ? mx : (pass == 2 ? my : mz)) + rad]);
    const double re = zdouble(acc.re), im = zdouble(acc.im);
    const double lr = pre * re - pim * im, li = pre * im + pim * re;
    const int ins = 80 * k + (pass == 0 ? e : 16 + 16 * (pass - 1) + e);
    double* o = out + (((size_t)ins * n_mom + m) * lt + t) * 2;
    if (accumulate) {
      o[0] += lr;
      o[1] += li;
    } else {
      o[0] = lr;
      o[1] = li;
    }
  }
}

// z transform of the partial sums of field precision R (FP32: float2 parts)
template <typename R>
int launch_z(const tsm_gauge* g, const void* part, const int* mom_dev, int n_mom, int rad, double mup, double* out,
             int accumulate, int unit_prefactor, cudaStream_t st) {
  using PT = typename PartOf<R>::type;
  using Z = typename ZReal<PT>::type;
  const int lz = g->geom.L[2], lt = g->geom.L[3], nx = 2 * rad + 1;
  const size_t zsmem = ((size_t)nx * lz + nx + lz) * sizeof(cplx<Z>);
  TSM_CUDA(cudaFuncSetAttribute(project_z_kernel<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsmem));
  count_launches(1);
  project_z_kernel<PT><<<z_grid(lt, n_mom), Z_BS, zsmem, st>>>(static_cast<const PT*>(part), mom_dev, n_mom, g->geom,
                                                               rad, mup, out, accumulate, unit_prefactor);
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

// ---------------------------------------------------------------- standard estimator (time dilution)
// For sources eta (a Z4 volume source, or one kept on a single timeslice:
// time dilution) and their solutions s = M(mu)^{-1} eta, the bilinear
// psibar(y) K psi(z) is estimated by eta(y)^dag K s(z) for the u flavour and,
// through g5-hermiticity, by conj(eta(z)^dag g5 K^dag g5 s(y)) for the d
// flavour.  Both come from the 4x4 matrices (no g5 factor)
//   M[a][b]     = sum_c conj(eta_ac(x)) s_bc(x)
//   D_mu[a][b]  = 1/4 sum_c [conj(eta_ac(x)) (U_mu(x) s(x+mu))_bc - conj(eta_ac(x+mu)) (U_mu(x)^dag s(x))_bc]
// (the derivative's backward terms are D_mu at x - mu, applied after the
// projection as in the one-end route), traced per site with Gamma_g (u) and
// with g5 Gamma_g^dag g5 (d) before any sum over sites, for the FP32
// accuracy reason given at the top of this file.  A source on timeslice t0
// touches M and the F part of D on t0 and the G part of D_t on t0 - 1 only.
template <typename R>
struct TdilArgs {
  Geom g;
  const void* s;
  const void* eta;
  const void* links;
  const int* t0;  // per source: its timeslice, or -1 for a volume source
  int nsrc;
  cplx<R>* F;     // [160][V]: pass * 32 + (0: u - d, 16: u + d) + g
};

template <typename R>
__device__ __forceinline__ void matvec_dag(cplx<R> (&w)[12], const cplx<R> (&u)[3][3], const cplx<R> (&p)[12], R sgn) {
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cplx<R> t = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; ++b) cmacc(t, u[b][a], p[3 * sp + b]);
      w[3 * sp + a] = sgn * t;
    }
}

template <typename R, int PS, int PL>
__global__ void __launch_bounds__(FLD_BS, sizeof(R) == 4 ? 3 : 1) tdil_fields_kernel(TdilArgs<R> a) {
  const int pass = blockIdx.x % 5;
  const int i = (blockIdx.x / 5) * FLD_BS + threadIdx.x;
  if (i >= a.g.V) return;
  const size_t V = (size_t)a.g.V;
  int c[4];
  site_coords(a.g, i, c);
  cplx<R> m[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) m[k] = mk<R>(0, 0);
  if (pass == 0) {
    for (int r = 0; r < a.nsrc; ++r) {
      const int t0 = a.t0[r];
      if (t0 >= 0 && t0 != c[3]) continue;
      cplx<R> e[12], x[12];
      SpinorIO<PS>::load(a.eta, V, r, i, e);
      SpinorIO<PS>::load(a.s, V, r, i, x);
      outer<false>(m, e, x);
    }
  } else {
    const int mu = pass - 1;
    const int nf = fwd_site_rt(a.g, i, c, mu);
    const int tn = (mu == 3) ? (c[3] + 1 == a.g.L[3] ? 0 : c[3] + 1) : c[3];
    cplx<R> u[3][3];
    LinkIO<PL>::load(a.links, V, mu, i, u);
    const R sf = (mu == 3 && c[3] == a.g.L[3] - 1) ? (R)a.g.bc : (R)1;
    for (int r = 0; r < a.nsrc; ++r) {
      const int t0 = a.t0[r];
      const bool f_on = t0 < 0 || t0 == c[3];
      const bool g_on = t0 < 0 || t0 == tn;
      cplx<R> e[12], x[12], w[12];
      if (f_on) {  // conj(eta(x)) (U(x) s(x+mu))
        SpinorIO<PS>::load(a.eta, V, r, i, e);
        SpinorIO<PS>::load(a.s, V, r, nf, x);
        matvec(w, u, x, sf);
        outer<false>(m, e, w);
      }
      if (g_on) {  // - conj(eta(x+mu)) (U(x)^dag s(x))
        SpinorIO<PS>::load(a.eta, V, r, nf, e);
        SpinorIO<PS>::load(a.s, V, r, i, x);
        matvec_dag(w, u, x, sf);
        outer<true>(m, e, w);
      }
    }
  }
  const R scale = pass ? (R)0.25 : (R)1;
  cplx<R>* out = a.F + (size_t)pass * 32 * V + i;
  store_std_traces(out, V, m, scale, pass ? (R)-1 : (R)1, std::make_integer_sequence<int, 16>{});
}


// Hopping parameter expansion of the ultra-local insertions: their loops
// come from the remainder field Y^4 s (A), plus the exact part of the first
// four orders, a constant per site, added at p = 0 once per source covering
// the timeslice (cnt[t] sources, Vs sites each); the derivative insertions
// keep the plain loops (B).
__global__ void hpe_merge_kernel(const double* __restrict__ A, const double* __restrict__ B,
                                 const double2* __restrict__ exact, const int* __restrict__ cnt, double vs, int m0,
                                 int n_mom, int lt, double* out, int accumulate) {
  const size_t n = (size_t)160 * n_mom * lt;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int ins = (int)(k / ((size_t)n_mom * lt));
  const int rem = (int)(k % ((size_t)n_mom * lt));
  const int m = rem / lt, t = rem % lt;
  double re, im;
  if ((ins % 80) < 16) {
    re = A[2 * k];
    im = A[2 * k + 1];
    if (m == m0) {
      re += cnt[t] * vs * exact[ins].x;
      im += cnt[t] * vs * exact[ins].y;
    }
  } else {
    re = B[2 * k];
    im = B[2 * k + 1];
  }
  if (accumulate) {
    out[2 * k] += re;
    out[2 * k + 1] += im;
  } else {
    out[2 * k] = re;
    out[2 * k + 1] = im;
  }
}

// Exact part of the hopping expansion per site for the 160 insertions (zero
// for the derivative ones): with A0^-1 = (1 - i mu' g5)/(1 + mu'^2) and
// P+-_mu = 1 +- g_mu, orders 0 and 2 (the only closed paths of length < 4
// when every extent is >= 4: x -> x +- mu -> x, where U U^dag = 1) give
//   c_u(Gamma) = 3 Tr_s[Gamma (A0^-1 + kappa^2 sum_mu (A0^-1 P- A0^-1 P+ A0^-1 + A0^-1 P+ A0^-1 P- A0^-1))]
// and the d flavour conj(c_u(g5 Gamma^dag g5)).
void hpe_exact(double kappa, double mu, HostCplx out[160]) {
  Mat4 g[4], a0i, one, inner, t1, t2;
  chiral_gammas(g);
  const double mup = 2.0 * kappa * mu, d = 1.0 + mup * mup;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      one[i][j] = HostCplx{i == j ? 1.0 : 0.0, 0.0};
      a0i[i][j] = HostCplx{0.0, 0.0};
    }
  for (int i = 0; i < 4; ++i) a0i[i][i] = HostCplx{1.0 / d, (i < 2 ? -mup : mup) / d};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) inner[i][j] = a0i[i][j];
  for (int m = 0; m < 4; ++m) {
    Mat4 pm, pp;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        pm[i][j] = HostCplx{one[i][j].re - g[m][i][j].re, one[i][j].im - g[m][i][j].im};
        pp[i][j] = HostCplx{one[i][j].re + g[m][i][j].re, one[i][j].im + g[m][i][j].im};
      }
    for (int order = 0; order < 2; ++order) {
      const Mat4* first = order == 0 ? &pm : &pp;
      const Mat4* second = order == 0 ? &pp : &pm;
      mat_mul(a0i, *first, t1);
      mat_mul(t1, a0i, t2);
      mat_mul(t2, *second, t1);
      mat_mul(t1, a0i, t2);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
          inner[i][j].re += kappa * kappa * t2[i][j].re;
          inner[i][j].im += kappa * kappa * t2[i][j].im;
        }
    }
  }
  HostCplx cu[16];
  Mat4 gam[16];
  for (int idx = 0; idx < 16; ++idx) {
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) gam[idx][i][j] = one[i][j];
    for (int bit = 0; bit < 4; ++bit)
      if ((idx >> bit) & 1) {
        mat_mul(gam[idx], g[bit], t1);
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) gam[idx][i][j] = t1[i][j];
      }
    mat_mul(gam[idx], inner, t1);
    double re = 0, im = 0;
    for (int i = 0; i < 4; ++i) {
      re += t1[i][i].re;
      im += t1[i][i].im;
    }
    cu[idx] = HostCplx{3.0 * re, 3.0 * im};
  }
  for (int i = 0; i < 160; ++i) out[i] = HostCplx{0.0, 0.0};
  for (int idx = 0; idx < 16; ++idx) {
    // g5 Gamma^dag g5 = sign * Gamma_k
    Mat4 gd;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const double s5 = ((i < 2) == (j < 2)) ? 1.0 : -1.0;
        gd[i][j] = HostCplx{s5 * gam[idx][j][i].re, -s5 * gam[idx][j][i].im};
      }
    int kk = -1;
    double sign = 0.0;
    for (int k = 0; k < 16 && kk < 0; ++k)
      for (double sg : {1.0, -1.0}) {
        double diff = 0.0;
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j)
            diff += fabs(gd[i][j].re - sg * gam[k][i][j].re) + fabs(gd[i][j].im - sg * gam[k][i][j].im);
        if (diff < 1e-9) {
          kk = k;
          sign = sg;
          break;
        }
      }
    const HostCplx dd{sign * cu[kk].re, -sign * cu[kk].im};  // conj(sign c_u(k))
    out[idx] = HostCplx{cu[idx].re - dd.re, cu[idx].im - dd.im};
    out[80 + idx] = HostCplx{cu[idx].re + dd.re, cu[idx].im + dd.im};
  }
}

}  // namespace

struct ContractWorkspace {
  std::mutex mu;  // held while a contraction enqueues its work
  UseOrder order;  // orders the GPU use across the callers' streams
  DevBuf v, fields, part, mom, aux, hpe;
};

void ContractWsDeleter::operator()(ContractWorkspace* w) const { delete w; }

namespace {

// staged planes, x results, y results, alignment, twiddle tables (cs bytes per complex value)
size_t xy_smem(const Geom& g, int rad, int nfc, size_t cs) {
  const int nx = 2 * rad + 1;
  return cs * ((size_t)nfc * g.L[1] * (g.L[0] + 1) + (size_t)nfc * g.L[1] * nx + (size_t)nx * nx * nfc +
               (size_t)nx * (g.L[0] + g.L[1])) + 16;
}

// Fields per block of the x/y transform: the largest of 8, 4, 2 dividing
// nfields whose shared memory stays within 64 KB (three or more blocks per
// SM), else a single field within the 227 KB a block may hold; 0 if none.
int xy_chunk(const Geom& g, int rad, size_t cs, int nfields) {
  for (int nfc : {8, 4, 2})
    if (nfields % nfc == 0 && xy_smem(g, rad, nfc, cs) <= 64 * 1024) return nfc;
  return xy_smem(g, rad, 1, cs) <= 227 * 1024 ? 1 : 0;
}

// x/y transform of nfields site fields of type cplx<R> into part
template <typename R>
int launch_xy(tsm_gauge* g, int rad, const void* F, int nfields, void* part, cudaStream_t st) {
  const int nfc = xy_chunk(g->geom, rad, sizeof(cplx<R>), nfields);
  if (nfc == 0)
    return fail(TSM_ERR_INVALID_ARG, "plane %dx%d too large for the contraction", g->geom.L[0], g->geom.L[1]);
  const size_t smem = xy_smem(g->geom, rad, nfc, sizeof(cplx<R>));
  auto kern = contract_xy_kernel<R>;
  TSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  count_launches(1);
  const unsigned nblk = (unsigned)(g->geom.L[2] * g->geom.L[3]) * (unsigned)(nfields / nfc);
  kern<<<nblk, XY_BS, smem, st>>>(static_cast<const cplx<R>*>(F), g->geom, rad, nfc, nfields,
                                  static_cast<typename PartOf<R>::type*>(part));
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

// Site fields then x/y transform; F holds 160 V fields of type cplx<R>.
template <typename R, int PS, int PL>
int launch_fields_xy(tsm_gauge* g, const void* s_dev, const void* v_dev, int nsrc, int rad, void* F, void* part,
                     cudaStream_t st, EventPair* ev_f, EventPair* ev_xy) {
  FieldArgs<R> a;
  a.g = g->geom;
  a.s = s_dev;
  a.v = v_dev;
  a.links = g->links[PL].p;
  a.nsrc = nsrc;
  a.F = static_cast<cplx<R>*>(F);
  const unsigned nblk = (unsigned)((g->geom.V + FLD_BS - 1) / FLD_BS);
  count_launches(1);
  if (ev_f) TSM_TRY(ev_f->begin(st));
  if constexpr (std::is_same<R, float>::value) {
    contract_fields_pairs_kernel<PS, PL><<<nblk * 5, FLD_BS, 0, st>>>(a);
  } else {
    contract_fields_kernel<R, PS, PL><<<nblk * 5, FLD_BS, 0, st>>>(a);
  }
  if (ev_f) TSM_TRY(ev_f->end(st));
  TSM_CUDA(cudaGetLastError());
  if (ev_xy) TSM_TRY(ev_xy->begin(st));
  TSM_TRY(launch_xy<R>(g, rad, a.F, 160, part, st));
  if (ev_xy) TSM_TRY(ev_xy->end(st));
  return TSM_OK;
}

}  // namespace

int prepare_contract(tsm_gauge* g, int prec, int nsrc, int n_mom, const int* mom_host, int slot, cudaStream_t st) {
  if (slot < 0 || slot > 1 || nsrc < 1) return fail(TSM_ERR_INVALID_ARG, "prepare_contract: slot %d, nsrc %d", slot, nsrc);
  if (prec != TSM_F32 && prec != TSM_F64) return fail(TSM_ERR_INVALID_ARG, "contraction precision %d", prec);
  int rad = 0;
  for (int m = 0; m < 3 * n_mom; ++m) rad = std::max(rad, std::abs(mom_host[m]));
  if (rad > 8) return fail(TSM_ERR_INVALID_ARG, "momentum component outside [-8, 8]");
  ContractWorkspace* wp;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    if (!g->contract_ws[slot]) g->contract_ws[slot].reset(new ContractWorkspace());
    wp = g->contract_ws[slot].get();
    if (!g->gamma_ready) {
      TSM_TRY(upload_gamma_table(st));
      g->gamma_ready = true;
    }
  }
  ContractWorkspace& w = *wp;
  {
    std::lock_guard<std::mutex> wlock(w.mu);
    const int V = g->geom.V, nx = 2 * rad + 1;
    const size_t cs = prec == TSM_F32 ? sizeof(cplx<float>) : sizeof(cplx<double>);
    TSM_TRY(w.order.enter(st));
    TSM_TRY(w.v.reserve((size_t)nsrc * spinor_chunks(prec) * V * 16));
    TSM_TRY(w.fields.reserve((size_t)160 * V * cs));
    TSM_TRY(w.part.reserve((size_t)g->geom.L[2] * g->geom.L[3] * 160 * nx * nx * sizeof(double2)));
    TSM_TRY(w.mom.reserve(sizeof(int) * 3 * (size_t)std::max(n_mom, 1)));
    TSM_TRY(w.order.leave(st));
  }
  int nr = 1;
  return tuned_nr(g, prec, prec, nsrc, st, &nr);
}

int contract_loops(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                   const int* mom_host, double* out_dev, int accumulate, cudaStream_t st, int slot) {
  if (slot < 0 || slot > 1) return fail(TSM_ERR_INVALID_ARG, "workspace slot %d", slot);
  if (prec != TSM_F32 && prec != TSM_F64)
    return fail(TSM_ERR_INVALID_ARG, "contraction takes F32 or F64 solutions, got precision %d", prec);
  if (!has_prec(g, prec)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", prec);
  int rad = 0;
  for (int m = 0; m < n_mom; ++m)
    for (int d = 0; d < 3; ++d) {
      const int n = mom_host[3 * m + d];
      if (n > 8 || n < -8) return fail(TSM_ERR_INVALID_ARG, "momentum component %d outside [-8, 8]", n);
      rad = std::max(rad, n < 0 ? -n : n);
    }
  ContractWorkspace* wp;
  {
    std::lock_guard<std::mutex> lock(g->mu);
    if (!g->contract_ws[slot]) g->contract_ws[slot].reset(new ContractWorkspace());
    wp = g->contract_ws[slot].get();
    if (!g->gamma_ready) {
      TSM_TRY(upload_gamma_table(st));
      g->gamma_ready = true;
    }
  }
  ContractWorkspace& w = *wp;
  std::lock_guard<std::mutex> wlock(w.mu);
  TSM_TRY(w.order.enter(st));
  const int V = g->geom.V;
  const int nx = 2 * rad + 1;
  const int lz = g->geom.L[2], lt = g->geom.L[3];
  const size_t cs = prec == TSM_F32 ? sizeof(cplx<float>) : sizeof(cplx<double>);
  TSM_TRY(w.v.reserve((size_t)nsrc * spinor_chunks(prec) * V * 16));
  TSM_TRY(w.fields.reserve((size_t)160 * V * cs));
  TSM_TRY(w.part.reserve((size_t)lz * lt * 160 * nx * nx * sizeof(double2)));
  TSM_TRY(w.mom.reserve(sizeof(int) * 3 * (size_t)std::max(n_mom, 1)));
  TSM_CUDA(cudaMemcpyAsync(w.mom.p, mom_host, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, st));
  const bool prof = profiling();
  EventPair ev_v, ev_f, ev_xy, ev_z;
  // v = g5 A s
  if (prof) TSM_TRY(ev_v.begin(st));
  TSM_TRY(dslash_apply_mixed(g, prec, prec, TSM_OP_A, kappa, 0.0, s_dev, w.v.p, nsrc, 1, st));
  if (prof) TSM_TRY(ev_v.end(st));
  if (prec == TSM_F32)
    TSM_TRY((launch_fields_xy<float, TSM_F32, TSM_F32>(g, s_dev, w.v.p, nsrc, rad, w.fields.p, w.part.as<double2>(),
                                                        st, prof ? &ev_f : nullptr, prof ? &ev_xy : nullptr)));
  else
    TSM_TRY((launch_fields_xy<double, TSM_F64, TSM_F64>(g, s_dev, w.v.p, nsrc, rad, w.fields.p,
                                                         w.part.as<double2>(), st, prof ? &ev_f : nullptr,
                                                         prof ? &ev_xy : nullptr)));
  if (prof) TSM_TRY(ev_z.begin(st));
  if (prec == TSM_F32)
    TSM_TRY(launch_z<float>(g, w.part.p, w.mom.as<int>(), n_mom, rad, 2.0 * kappa * mu, out_dev, accumulate, 0, st));
  else
    TSM_TRY(launch_z<double>(g, w.part.p, w.mom.as<int>(), n_mom, rad, 2.0 * kappa * mu, out_dev, accumulate, 0, st));
  if (prof) TSM_TRY(ev_z.end(st));
  if (prof) {
    const double v = (double)V, n = (double)nsrc, b = spinor_site_bytes(prec), l = link_site_bytes(prec);
    const double part_bytes = (double)lz * lt * nx * nx * 160 * (prec == TSM_F32 ? 8 : 16);
    const double field_bytes = 160.0 * v * (double)cs;
    const double out_bytes = 160.0 * n_mom * lt * 16 * (accumulate ? 2 : 1);
    const char* pn = prec == TSM_F32 ? "f32" : "f64";
    char name[48];
    snprintf(name, sizeof(name), "contract_g5A_%s", pn);
    prof_add(name, ev_v.seconds(), v * (l + 2 * n * b), v * n * 1392.0);
    // per site and source: 4 x (2 colour matvecs x 4 spins + 3 outer products) + 2 outer products
    const double cmac_src = 4 * (2 * 36 + 3 * 48) + 2 * 48;
    snprintf(name, sizeof(name), "contract_fields_%s", pn);
    prof_add(name, ev_f.seconds(), v * (l + 2 * n * b) + field_bytes, 8.0 * v * n * cmac_src);
    // x transform of 160 fields (nx momenta) + y transform (nx^2 momenta, per row)
    const double cmac_dft = 160.0 * nx + 160.0 * nx * nx / g->geom.L[0];
    snprintf(name, sizeof(name), "contract_xy_%s", pn);
    prof_add(name, ev_xy.seconds(), field_bytes + part_bytes, 8.0 * v * cmac_dft);
    snprintf(name, sizeof(name), "contract_project_z");
    prof_add(name, ev_z.seconds(), part_bytes + out_bytes, 8.0 * 160.0 * n_mom * lt * lz + 8.0 * 160 * n_mom * lt);
  }
  return w.order.leave(st);
}


namespace {

int contract_ws_slot(tsm_gauge* g, int slot, ContractWorkspace** out, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g->mu);
  if (!g->contract_ws[slot]) g->contract_ws[slot].reset(new ContractWorkspace());
  *out = g->contract_ws[slot].get();
  if (!g->gamma_ready) {
    TSM_TRY(upload_gamma_table(st));
    g->gamma_ready = true;
  }
  return TSM_OK;
}

int tdil_body(tsm_gauge* g, ContractWorkspace& w, int prec, const void* s_dev, const void* eta_dev, int nsrc,
              const std::vector<int>& t0, int rad, int n_mom, const int* mom_host,
              double* out_dev, int accumulate, cudaStream_t st);

// argument checks shared by the standard-estimator entries: per-source
// timeslices and the momentum radius
int tdil_setup(const tsm_gauge* g, int prec, int nsrc, const int* t0_host, int n_mom, const int* mom_host,
               std::vector<int>& t0, int& rad) {
  if (prec != TSM_F32 && prec != TSM_F64)
    return fail(TSM_ERR_INVALID_ARG, "contraction takes F32 or F64 fields, got precision %d", prec);
  if (!has_prec(g, prec)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", prec);
  const int lt = g->geom.L[3];
  t0.assign(nsrc, -1);
  if (t0_host)
    for (int r = 0; r < nsrc; ++r) {
      if (t0_host[r] < -1 || t0_host[r] >= lt) return fail(TSM_ERR_INVALID_ARG, "source %d: timeslice %d", r, t0_host[r]);
      t0[r] = t0_host[r];
    }
  rad = 0;
  for (int m = 0; m < n_mom; ++m)
    for (int d = 0; d < 3; ++d) {
      const int n = mom_host[3 * m + d];
      if (n > 8 || n < -8) return fail(TSM_ERR_INVALID_ARG, "momentum component %d outside [-8, 8]", n);
      rad = std::max(rad, n < 0 ? -n : n);
    }
  return TSM_OK;
}

}  // namespace

int contract_tdil(tsm_gauge* g, int prec, const void* s_dev, const void* eta_dev, int nsrc, const int* t0_host,
                  int n_mom, const int* mom_host, double* out_dev, int accumulate, cudaStream_t st) {
  std::vector<int> t0;
  int rad = 0;
  TSM_TRY(tdil_setup(g, prec, nsrc, t0_host, n_mom, mom_host, t0, rad));
  ContractWorkspace* wp;
  TSM_TRY(contract_ws_slot(g, 0, &wp, st));
  std::lock_guard<std::mutex> wlock(wp->mu);
  TSM_TRY(wp->order.enter(st));
  TSM_TRY(tdil_body(g, *wp, prec, s_dev, eta_dev, nsrc, t0, rad, n_mom, mom_host, out_dev, accumulate, st));
  return wp->order.leave(st);
}

namespace {

int tdil_body(tsm_gauge* g, ContractWorkspace& w, int prec, const void* s_dev, const void* eta_dev, int nsrc,
              const std::vector<int>& t0, int rad, int n_mom, const int* mom_host,
              double* out_dev, int accumulate, cudaStream_t st) {
  const int V = g->geom.V;
  const int lt = g->geom.L[3];
  const int nx = 2 * rad + 1;
  const int lz = g->geom.L[2];
  const size_t cs = prec == TSM_F32 ? sizeof(cplx<float>) : sizeof(cplx<double>);
  TSM_TRY(w.fields.reserve((size_t)160 * V * cs));
  TSM_TRY(w.part.reserve((size_t)lz * lt * 160 * nx * nx * sizeof(double2)));
  TSM_TRY(w.mom.reserve(sizeof(int) * 3 * (size_t)n_mom));
  TSM_TRY(w.aux.reserve(sizeof(int) * (size_t)nsrc));
  int* t0_dev = w.aux.as<int>();
  TSM_CUDA(cudaMemcpyAsync(w.mom.p, mom_host, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, st));
  TSM_CUDA(cudaMemcpyAsync(t0_dev, t0.data(), sizeof(int) * nsrc, cudaMemcpyHostToDevice, st));
  const unsigned nblk = (unsigned)((V + FLD_BS - 1) / FLD_BS);
  count_launches(1);
  if (prec == TSM_F32) {
    TdilArgs<float> a{g->geom, s_dev, eta_dev, g->links[TSM_F32].p, t0_dev, nsrc, w.fields.as<cplx<float>>()};
    tdil_fields_kernel<float, TSM_F32, TSM_F32><<<nblk * 5, FLD_BS, 0, st>>>(a);
    TSM_CUDA(cudaGetLastError());
    TSM_TRY(launch_xy<float>(g, rad, w.fields.p, 160, w.part.as<double2>(), st));
  } else {
    TdilArgs<double> a{g->geom, s_dev, eta_dev, g->links[TSM_F64].p, t0_dev, nsrc, w.fields.as<cplx<double>>()};
    tdil_fields_kernel<double, TSM_F64, TSM_F64><<<nblk * 5, FLD_BS, 0, st>>>(a);
    TSM_CUDA(cudaGetLastError());
    TSM_TRY(launch_xy<double>(g, rad, w.fields.p, 160, w.part.as<double2>(), st));
  }
  // the fields carry their flavour factors already: unit prefactors
  if (prec == TSM_F32) return launch_z<float>(g, w.part.p, w.mom.as<int>(), n_mom, rad, 0.0, out_dev, accumulate, 1, st);
  return launch_z<double>(g, w.part.p, w.mom.as<int>(), n_mom, rad, 0.0, out_dev, accumulate, 1, st);
}

}  // namespace

int contract_hpe(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, const void* eta_dev, int nsrc,
                 const int* t0_host, int n_mom, const int* mom_host, double* out_dev, int accumulate,
                 cudaStream_t st) {
  for (int d = 0; d < 4; ++d)
    if (g->geom.L[d] < 4) return fail(TSM_ERR_INVALID_ARG, "the expansion's exact part needs every extent >= 4");
  std::vector<int> t0;
  int rad = 0;
  TSM_TRY(tdil_setup(g, prec, nsrc, t0_host, n_mom, mom_host, t0, rad));
  const int lt = g->geom.L[3];
  int m0 = -1;
  for (int m = 0; m < n_mom; ++m)
    if (mom_host[3 * m] == 0 && mom_host[3 * m + 1] == 0 && mom_host[3 * m + 2] == 0) m0 = m;
  std::vector<int> cnt(lt, 0);
  for (int r = 0; r < nsrc; ++r) {
    if (t0[r] < 0)
      for (int t = 0; t < lt; ++t) ++cnt[t];
    else
      ++cnt[t0[r]];
  }
  HostCplx ex[160];
  hpe_exact(kappa, mu, ex);
  ContractWorkspace* wp;
  TSM_TRY(contract_ws_slot(g, 0, &wp, st));
  ContractWorkspace& w = *wp;
  std::lock_guard<std::mutex> wlock(w.mu);
  TSM_TRY(w.order.enter(st));
  const size_t fs = (size_t)nsrc * spinor_chunks(prec) * g->geom.V * 16;
  const size_t n_out = (size_t)160 * n_mom * lt * 2;
  const size_t bytes = 2 * fs + 2 * n_out * sizeof(double) + 160 * sizeof(double2) + (size_t)lt * sizeof(int);
  TSM_TRY(w.hpe.reserve(bytes));
  char* base = w.hpe.as<char>();
  void* ya = base;
  void* yb = base + fs;
  double* tmp_a = reinterpret_cast<double*>(base + 2 * fs);
  double* tmp_b = tmp_a + n_out;
  double2* ex_dev = reinterpret_cast<double2*>(tmp_b + n_out);
  int* cnt_dev = reinterpret_cast<int*>(ex_dev + 160);
  // Y = A0^-1 kappa H = (h0 + i h1 g5) H,  h0 + i h1 g5 = kappa (1 - i mu' g5) / (1 + mu'^2)
  const double mup = 2.0 * kappa * mu, dd = 1.0 + mup * mup;
  const double h0 = kappa / dd, h1 = -kappa * mup / dd;
  TSM_TRY(hop_general(g, prec, s_dev, nullptr, ya, nsrc, 0.0, 0.0, h0, h1, st));
  TSM_TRY(hop_general(g, prec, ya, nullptr, yb, nsrc, 0.0, 0.0, h0, h1, st));
  TSM_TRY(hop_general(g, prec, yb, nullptr, ya, nsrc, 0.0, 0.0, h0, h1, st));
  TSM_TRY(hop_general(g, prec, ya, nullptr, yb, nsrc, 0.0, 0.0, h0, h1, st));
  TSM_TRY(tdil_body(g, w, prec, yb, eta_dev, nsrc, t0, rad, n_mom, mom_host, tmp_a, 0, st));
  TSM_TRY(tdil_body(g, w, prec, s_dev, eta_dev, nsrc, t0, rad, n_mom, mom_host, tmp_b, 0, st));
  std::vector<double2> exh(160);
  for (int i = 0; i < 160; ++i) exh[i] = make_double2(ex[i].re, ex[i].im);
  TSM_CUDA(cudaMemcpyAsync(ex_dev, exh.data(), sizeof(double2) * 160, cudaMemcpyHostToDevice, st));
  TSM_CUDA(cudaMemcpyAsync(cnt_dev, cnt.data(), sizeof(int) * lt, cudaMemcpyHostToDevice, st));
  const double vs = (double)g->geom.L[0] * g->geom.L[1] * g->geom.L[2];
  const size_t n = (size_t)160 * n_mom * lt;
  count_launches(1);
  hpe_merge_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tmp_a, tmp_b, ex_dev, cnt_dev, vs, m0, n_mom, lt,
                                                                 out_dev, accumulate);
  TSM_CUDA(cudaGetLastError());
  return w.order.leave(st);  // pageable sources of the copies above are staged before the calls return
}
}  // namespace tsm

// ---------------------------------------------------------------- allocation-free variant
// For callers that must not allocate device memory during a call -- code that
// runs while a memory pool or a graph capture forbids cudaMalloc, or
// latency-bound loops where an allocation would synchronise the device --
// the contraction can run entirely in a fixed scratch region compiled into
// the library.  Every device that loads the library holds this array until
// the process exits.  All calls on a device share it, so calls that overlap
// on the GPU race; nothing in it needs to start at zero (each launch writes
// every scratch word it later reads).
static __device__ __align__(256) unsigned char g_contract_scratch[TSM_CONTRACT_NOALLOC_MAX_BYTES];

namespace tsm {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {nullptr};

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }

// Host-side address of the scratch array on `dev` (which must be current);
// looked up, together with the Gamma table upload, on the first call per device.
int noalloc_setup(int dev, unsigned char** out, cudaStream_t st) {
  if (dev < 0 || dev >= kMaxDevices) return fail(TSM_ERR_INVALID_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> l(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_contract_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    TSM_TRY(upload_gamma_table(st));
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return TSM_OK;
}
}  // namespace

int contract_loops_noalloc(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                           const int* mom_host, double* out_dev, int accumulate, cudaStream_t st) {
  if (prec != TSM_F32 && prec != TSM_F64)
    return fail(TSM_ERR_INVALID_ARG, "contraction takes F32 or F64 solutions, got precision %d", prec);
  if (!has_prec(g, prec)) return fail(TSM_ERR_INVALID_ARG, "gauge has no copy in precision %d", prec);
  int rad = 0;
  for (int m = 0; m < n_mom; ++m)
    for (int d = 0; d < 3; ++d) {
      const int n = mom_host[3 * m + d];
      if (n > 8 || n < -8) return fail(TSM_ERR_INVALID_ARG, "momentum component %d outside [-8, 8]", n);
      rad = std::max(rad, n < 0 ? -n : n);
    }
  const int V = g->geom.V;
  const int nx = 2 * rad + 1;
  const int lz = g->geom.L[2], lt = g->geom.L[3];
  const size_t cs = prec == TSM_F32 ? sizeof(cplx<float>) : sizeof(cplx<double>);
  const size_t mom_bytes = round256(sizeof(int) * 3 * (size_t)n_mom);
  const size_t v_bytes = round256((size_t)nsrc * spinor_chunks(prec) * V * 16);
  const size_t f_bytes = round256((size_t)160 * V * cs);
  const size_t part_bytes = round256((size_t)lz * lt * 160 * nx * nx * cs);  // float2 / double2 partials
  const size_t need = mom_bytes + v_bytes + f_bytes + part_bytes;
  if (need > (size_t)TSM_CONTRACT_NOALLOC_MAX_BYTES)
    return fail(TSM_ERR_INVALID_ARG,
                "tsm_contract_loops_noalloc needs %zu scratch bytes (solutions %zu + site fields %zu + partial sums "
                "%zu), above the fixed %d; use fewer sources per call, a smaller momentum radius or "
                "tsm_contract_loops",
                need, v_bytes, f_bytes, part_bytes, (int)TSM_CONTRACT_NOALLOC_MAX_BYTES);
  unsigned char* base = nullptr;
  TSM_TRY(noalloc_setup(g->ctx->device, &base, st));
  int* mom_dev = reinterpret_cast<int*>(base);
  void* v_dev = base + mom_bytes;
  void* f_dev = base + mom_bytes + v_bytes;
  double2* part = reinterpret_cast<double2*>(base + mom_bytes + v_bytes + f_bytes);
  TSM_CUDA(cudaMemcpyAsync(mom_dev, mom_host, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, st));
  TSM_TRY(dslash_apply_fixed(g, prec, TSM_OP_A, kappa, 0.0, s_dev, v_dev, nsrc, 1, 1, st));
  if (prec == TSM_F32)
    TSM_TRY((launch_fields_xy<float, TSM_F32, TSM_F32>(g, s_dev, v_dev, nsrc, rad, f_dev, part, st, nullptr,
                                                        nullptr)));
  else
    TSM_TRY((launch_fields_xy<double, TSM_F64, TSM_F64>(g, s_dev, v_dev, nsrc, rad, f_dev, part, st, nullptr,
                                                         nullptr)));
  if (prec == TSM_F32) return launch_z<float>(g, part, mom_dev, n_mom, rad, 2.0 * kappa * mu, out_dev, accumulate, 0, st);
  return launch_z<double>(g, part, mom_dev, n_mom, rad, 2.0 * kappa * mu, out_dev, accumulate, 0, st);
}

}  // namespace tsm
