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
// outer products because U commutes with g5), i.e. 10 x 16 = 160 complex
// fields per site, summed over the sources of the batch.  These fields are
// projected to momenta with a separable transform, x then y inside a
// (z, t)-plane block (FP32, short sums), and z in FP64 by a second kernel,
// which also forms every Gamma insertion from the projected 4x4 matrix
// ("by transposition and multiplication", Sec. 2.2):
//   L_g = pref_k sum_ab Gamma_g[a][b] D[a][b],   pref_0 = -2 i mu', pref_1 = 2.
// Gamma_g is a monomial matrix in the chiral basis, so each L_g is 4 terms.
#include <math.h>
#include <stdio.h>

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

constexpr int NF = 32;       // fields per pass: 2 flavour structures x 16
constexpr int K4_BS = 256;
constexpr int Z_BS = 256;

template <typename R>
struct ContractArgs {
  Geom g;
  const void* s;
  const void* v;
  const void* links;
  int nsrc;
  int rad;  // max |n_i|
  int nx;   // 2 rad + 1
  int rb;   // rows per row block
  double2* part;  // [Lz*T][nx*nx][160]
};

template <typename R>
__device__ __forceinline__ void matvec(cplx<R> (&w)[12], const cplx<R> (&u)[3][3], const cplx<R> (&p)[12],
                                       bool dag, R sgn) {
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

// acc[a*4+b] += g_a * scale * sum_c conj(l_ac) r_bc
template <typename R>
__device__ __forceinline__ void outer(cplx<R>* acc, const cplx<R> (&l)[12], const cplx<R> (&r)[12], R scale) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const R ga = (a < 2 ? scale : -scale);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      cplx<R> t = mk<R>(0, 0);
#pragma unroll
      for (int c = 0; c < 3; ++c) cmacc(t, l[3 * a + c], r[3 * b + c]);
      acc[4 * a + b] = acc[4 * a + b] + ga * t;
    }
  }
}

// Fields of pass P at site i, summed over the sources: 32 complex.
template <typename R, int PS, int PL>
__device__ void site_fields(cplx<R> (&acc)[NF], const ContractArgs<R>& a, int pass, int i, const int c[4]) {
#pragma unroll
  for (int f = 0; f < NF; ++f) acc[f] = mk<R>(0, 0);
  const size_t V = (size_t)a.g.V;
  if (pass == 0) {
    for (int r = 0; r < a.nsrc; ++r) {
      cplx<R> s0[12], v0[12];
      SpinorIO<PS>::load(a.s, V, r, i, s0);
      SpinorIO<PS>::load(a.v, V, r, i, v0);
      outer(acc, s0, s0, (R)1);
      outer(acc + 16, s0, v0, (R)1);
    }
    return;
  }
  const int mu = pass - 1;
  const int stride = dir_stride(a.g, mu);
  const int nf = fwd_site(a.g, i, c, mu, stride);
  const int nb = bwd_site(a.g, i, c, mu, stride);
  cplx<R> uf[3][3], ub[3][3];
  LinkIO<PL>::load(a.links, V, mu, i, uf);
  LinkIO<PL>::load(a.links, V, mu, nb, ub);
  const R sf = (mu == 3 && c[3] == a.g.L[3] - 1) ? (R)a.g.bc : (R)1;
  const R sb = (mu == 3 && c[3] == 0) ? (R)a.g.bc : (R)1;
  const R q = (R)0.25;
  for (int r = 0; r < a.nsrc; ++r) {
    cplx<R> t[12], w0[12], w1[12], s0[12];
    SpinorIO<PS>::load(a.s, V, r, nf, t);
    matvec(w0, uf, t, false, sf);
    SpinorIO<PS>::load(a.s, V, r, nb, t);
    matvec(w1, ub, t, true, sb);
#pragma unroll
    for (int k = 0; k < 12; ++k) w0[k] = w0[k] - w1[k];  // W^0
    SpinorIO<PS>::load(a.v, V, r, nf, t);
    matvec(w1, uf, t, false, sf);
    cplx<R> tb[12];
    SpinorIO<PS>::load(a.v, V, r, nb, t);
    matvec(tb, ub, t, true, sb);
#pragma unroll
    for (int k = 0; k < 12; ++k) w1[k] = w1[k] - tb[k];  // W^1
    SpinorIO<PS>::load(a.s, V, r, i, s0);
    outer(acc, s0, w0, q);
    outer(acc, w0, s0, -q);
    outer(acc + 16, s0, w1, q);
    SpinorIO<PS>::load(a.v, V, r, i, t);
    outer(acc + 16, w0, t, -q);
  }
}

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

// One block per (z, t) plane: fields -> x transform -> y transform -> part.
// Shared layouts keep the field index f fastest so that a warp touches
// consecutive words; F rows are padded by one element against bank conflicts.
constexpr int FSTR = NF + 1;

template <typename R, int PS, int PL>
__global__ void __launch_bounds__(K4_BS) contract_plane_kernel(ContractArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lx = a.g.L[0], ly = a.g.L[1], lz = a.g.L[2];
  const int plane = blockIdx.x;  // z + Lz * t
  const int z = plane % lz, t = plane / lz;
  const int nx = a.nx, nxy = nx * nx, rb = a.rb;
  cplx<R>* F = reinterpret_cast<cplx<R>*>(smem_raw);  // [rb*lx][FSTR]
  cplx<R>* X = F + (size_t)rb * lx * FSTR;            // [rb][nx][NF]
  cplx<R>* Y = X + (size_t)rb * nx * NF;              // [nxy][NF]
  cplx<R>* twx = Y + (size_t)nxy * NF;                // [nx][lx]
  cplx<R>* twy = twx + (size_t)nx * lx;               // [nx][ly]
  for (int k = threadIdx.x; k < nx * lx; k += blockDim.x) {
    const int n = k / lx - a.rad, x = k % lx;
    twiddle(twx[k], ((n * x) % lx + lx) % lx, lx);
  }
  for (int k = threadIdx.x; k < nx * ly; k += blockDim.x) {
    const int n = k / ly - a.rad, y = k % ly;
    twiddle(twy[k], ((n * y) % ly + ly) % ly, ly);
  }
  for (int pass = 0; pass < 5; ++pass) {
    for (int k = threadIdx.x; k < NF * nxy; k += blockDim.x) Y[k] = mk<R>(0, 0);
    for (int y0 = 0; y0 < ly; y0 += rb) {
      const int rows = min(rb, ly - y0);
      __syncthreads();
      for (int sidx = threadIdx.x; sidx < rows * lx; sidx += blockDim.x) {
        const int x = sidx % lx, y = y0 + sidx / lx;
        const int c[4] = {x, y, z, t};
        const int i = x + lx * (y + ly * (z + lz * t));
        cplx<R> acc[NF];
        site_fields<R, PS, PL>(acc, a, pass, i, c);
#pragma unroll
        for (int f = 0; f < NF; ++f) F[(size_t)sidx * FSTR + f] = acc[f];
      }
      __syncthreads();
      // x transform: X[row][n][f] = sum_x F[row*lx + x][f] e^{-2 pi i n x / lx}
      for (int k = threadIdx.x; k < NF * rows * nx; k += blockDim.x) {
        const int f = k % NF, rn = k / NF, n = rn % nx, row = rn / nx;
        cplx<R> sum = mk<R>(0, 0);
        for (int x = 0; x < lx; ++x) cmac(sum, F[((size_t)row * lx + x) * FSTR + f], twx[n * lx + x]);
        X[((size_t)row * nx + n) * NF + f] = sum;
      }
      __syncthreads();
      // y transform, accumulated over row blocks: Y[(n_x, n_y)][f]
      for (int k = threadIdx.x; k < NF * nxy; k += blockDim.x) {
        const int f = k % NF, nn = k / NF, n_x = nn / nx, n_y = nn % nx;
        cplx<R> sum = Y[k];
        for (int row = 0; row < rows; ++row)
          cmac(sum, X[((size_t)row * nx + n_x) * NF + f], twy[n_y * ly + y0 + row]);
        Y[k] = sum;
      }
    }
    __syncthreads();
    // part layout [plane][nxy][160]
    for (int k = threadIdx.x; k < NF * nxy; k += blockDim.x) {
      const int f = k % NF, nn = k / NF;
      a.part[((size_t)plane * nxy + nn) * 160 + pass * NF + f] = make_double2((double)Y[k].re, (double)Y[k].im);
    }
    __syncthreads();
  }
}

// z transform (FP64) and Gamma insertions.  Block (t, group): group = 2 pass + k
// holds one 4x4 matrix field (16 fields).
__global__ void __launch_bounds__(Z_BS) project_z_kernel(const double2* __restrict__ part, const int* __restrict__ mom,
                                                         int n_mom, int lz, int lt, int rad, int nx, double mup,
                                                         double* out, int accumulate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int t = blockIdx.x, group = blockIdx.y;
  const int pass = group >> 1, k = group & 1;
  const int nxy = nx * nx;
  double2* zs = reinterpret_cast<double2*>(smem_raw);  // [n_mom][16]
  double2* twz = zs + (size_t)n_mom * 16;               // [nx][lz]
  for (int q = threadIdx.x; q < nx * lz; q += blockDim.x) {
    const int n = q / lz - rad, zz = q % lz;
    double sn, cs;
    sincospi(2.0 * (double)(((n * zz) % lz + lz) % lz) / (double)lz, &sn, &cs);
    twz[q] = make_double2(cs, -sn);
  }
  __syncthreads();
  const int field0 = pass * NF + k * 16;
  for (int q = threadIdx.x; q < n_mom * 16; q += blockDim.x) {
    const int m = q / 16, e = q % 16;
    const int mx = mom[3 * m], my = mom[3 * m + 1], mz = mom[3 * m + 2];
    const int nn = (mx + rad) * nx + (my + rad);
    double re = 0.0, im = 0.0;
    for (int zz = 0; zz < lz; ++zz) {
      const double2 p = part[((size_t)(zz + lz * t) * nxy + nn) * 160 + field0 + e];
      const double2 w = twz[(mz + rad) * lz + zz];
      re += p.x * w.x - p.y * w.y;
      im += p.x * w.y + p.y * w.x;
    }
    zs[q] = make_double2(re, im);
  }
  __syncthreads();
  // prefactor: k = 0 -> -2 i mu', k = 1 -> 2
  const double pre = (k == 0) ? 0.0 : 2.0, pim = (k == 0) ? -2.0 * mup : 0.0;
  for (int q = threadIdx.x; q < n_mom * 16; q += blockDim.x) {
    const int m = q / 16, gi = q % 16;
    double re = 0.0, im = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int b = c_gamma.col[gi][a];
      const double gr = c_gamma.re[gi][a], gm = c_gamma.im[gi][a];
      const double2 d = zs[m * 16 + 4 * a + b];
      re += gr * d.x - gm * d.y;
      im += gr * d.y + gm * d.x;
    }
    const double lr = pre * re - pim * im, li = pre * im + pim * re;
    const int ins = 80 * k + (pass == 0 ? gi : 16 + 16 * (pass - 1) + gi);
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

}  // namespace

struct ContractWorkspace {
  DevBuf v, part, mom;
  bool gamma_ready = false;
};

void ContractWsDeleter::operator()(ContractWorkspace* w) const { delete w; }

namespace {

template <typename R, int PS, int PL>
int launch_planes(tsm_gauge* g, const void* s_dev, const void* v_dev, int nsrc, int rad, double2* part,
                  cudaStream_t st) {
  ContractArgs<R> a;
  a.g = g->geom;
  a.s = s_dev;
  a.v = v_dev;
  a.links = g->links[PL].p;
  a.nsrc = nsrc;
  a.rad = rad;
  a.nx = 2 * rad + 1;
  a.part = part;
  const int lx = g->geom.L[0], ly = g->geom.L[1];
  const size_t cs = sizeof(cplx<R>);
  const size_t fixed = (size_t)NF * a.nx * a.nx * cs + (size_t)a.nx * (lx + ly) * cs;
  const size_t per_row = (size_t)lx * FSTR * cs + (size_t)NF * a.nx * cs;
  const size_t budget = 160 * 1024;
  if (fixed + per_row > budget) return fail(TSM_ERR_INVALID_ARG, "plane %dx%d too large for the contraction", lx, ly);
  int rb_max = (int)std::min<size_t>((size_t)ly, (budget - fixed) / per_row);
  const int nrb = (ly + rb_max - 1) / rb_max;
  a.rb = (ly + nrb - 1) / nrb;
  const size_t smem = fixed + per_row * a.rb;
  auto kern = contract_plane_kernel<R, PS, PL>;
  TSM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  count_launches(1);
  kern<<<g->geom.L[2] * g->geom.L[3], K4_BS, smem, st>>>(a);
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

}  // namespace

int contract_loops(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
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
  std::lock_guard<std::mutex> lock(g->mu);
  if (!g->contract_ws) g->contract_ws.reset(new ContractWorkspace());
  ContractWorkspace& w = *g->contract_ws;
  if (!w.gamma_ready) {
    GammaTable t;
    TSM_TRY(build_gamma_table(t));
    TSM_CUDA(cudaMemcpyToSymbol(c_gamma, &t, sizeof(t)));
    w.gamma_ready = true;
  }
  const int V = g->geom.V;
  const int nx = 2 * rad + 1;
  const int lz = g->geom.L[2], lt = g->geom.L[3];
  TSM_TRY(w.v.reserve((size_t)nsrc * spinor_chunks(prec) * V * 16));
  TSM_TRY(w.part.reserve((size_t)lz * lt * 160 * nx * nx * sizeof(double2)));
  TSM_TRY(w.mom.reserve(sizeof(int) * 3 * (size_t)std::max(n_mom, 1)));
  TSM_CUDA(cudaMemcpyAsync(w.mom.p, mom_host, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, st));
  const bool prof = profiling();
  EventPair ev_v, ev_p, ev_z;
  // v = g5 A s
  if (prof) TSM_TRY(ev_v.begin(st));
  TSM_TRY(dslash_apply_mixed(g, prec, prec, TSM_OP_A, kappa, 0.0, s_dev, w.v.p, nsrc, 1, st));
  if (prof) TSM_TRY(ev_v.end(st));
  if (prof) TSM_TRY(ev_p.begin(st));
  if (prec == TSM_F32)
    TSM_TRY((launch_planes<float, TSM_F32, TSM_F32>(g, s_dev, w.v.p, nsrc, rad, w.part.as<double2>(), st)));
  else
    TSM_TRY((launch_planes<double, TSM_F64, TSM_F64>(g, s_dev, w.v.p, nsrc, rad, w.part.as<double2>(), st)));
  if (prof) TSM_TRY(ev_p.end(st));
  const size_t zsmem = (size_t)n_mom * 16 * sizeof(double2) + (size_t)nx * lz * sizeof(double2);
  TSM_CUDA(cudaFuncSetAttribute(project_z_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsmem));
  if (prof) TSM_TRY(ev_z.begin(st));
  count_launches(1);
  project_z_kernel<<<dim3(lt, 10), Z_BS, zsmem, st>>>(w.part.as<double2>(), w.mom.as<int>(), n_mom, lz, lt, rad, nx,
                                                      2.0 * kappa * mu, out_dev, accumulate);
  if (prof) TSM_TRY(ev_z.end(st));
  TSM_CUDA(cudaGetLastError());
  if (prof) {
    const double v = (double)V, n = (double)nsrc, b = spinor_site_bytes(prec), l = link_site_bytes(prec);
    const double part_bytes = (double)lz * lt * nx * nx * 160 * 16;
    const double out_bytes = 160.0 * n_mom * lt * 16 * (accumulate ? 2 : 1);
    const char* pn = prec == TSM_F32 ? "f32" : "f64";
    char name[48];
    snprintf(name, sizeof(name), "contract_g5A_%s", pn);
    prof_add(name, ev_v.seconds(), v * (l + 2 * n * b), v * n * 1392.0);
    // per site and source: 4 x (4 colour matvecs x 4 spins + 4 outer products) + 2 outer products;
    // per site and batch: x transform of 160 fields + y transform share
    const double cmac_src = 4 * (16 * 9 + 4 * 48) + 2 * 48;
    const double cmac_dft = 160.0 * nx + 160.0 * nx * nx / g->geom.L[0];
    snprintf(name, sizeof(name), "contract_plane_%s", pn);
    prof_add(name, ev_p.seconds(), v * (l + 2 * n * b) + part_bytes, 8.0 * v * (n * cmac_src + cmac_dft));
    snprintf(name, sizeof(name), "contract_project_z");
    prof_add(name, ev_z.seconds(), part_bytes + out_bytes, 8.0 * 160.0 * n_mom * lt * lz + 8.0 * 160 * n_mom * lt);
  }
  return TSM_OK;
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
int noalloc_setup(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(TSM_ERR_INVALID_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> l(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_contract_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
    GammaTable t;
    TSM_TRY(build_gamma_table(t));
    TSM_CUDA(cudaMemcpyToSymbol(c_gamma, &t, sizeof(t)));
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
  const size_t mom_bytes = round256(sizeof(int) * 3 * (size_t)n_mom);
  const size_t v_bytes = round256((size_t)nsrc * spinor_chunks(prec) * V * 16);
  const size_t part_bytes = round256((size_t)lz * lt * 160 * nx * nx * sizeof(double2));
  const size_t need = mom_bytes + v_bytes + part_bytes;
  if (need > (size_t)TSM_CONTRACT_NOALLOC_MAX_BYTES)
    return fail(TSM_ERR_INVALID_ARG,
                "tsm_contract_loops_noalloc needs %zu scratch bytes (fields %zu + partial sums %zu), above the "
                "fixed %d; use fewer sources per call, a smaller momentum radius or tsm_contract_loops",
                need, v_bytes, part_bytes, (int)TSM_CONTRACT_NOALLOC_MAX_BYTES);
  unsigned char* base = nullptr;
  TSM_TRY(noalloc_setup(g->ctx->device, &base));
  int* mom_dev = reinterpret_cast<int*>(base);
  void* v_dev = base + mom_bytes;
  double2* part = reinterpret_cast<double2*>(base + mom_bytes + v_bytes);
  TSM_CUDA(cudaMemcpyAsync(mom_dev, mom_host, sizeof(int) * 3 * n_mom, cudaMemcpyHostToDevice, st));
  TSM_TRY(dslash_apply_fixed(g, prec, TSM_OP_A, kappa, 0.0, s_dev, v_dev, nsrc, 1, 1, st));
  if (prec == TSM_F32)
    TSM_TRY((launch_planes<float, TSM_F32, TSM_F32>(g, s_dev, v_dev, nsrc, rad, part, st)));
  else
    TSM_TRY((launch_planes<double, TSM_F64, TSM_F64>(g, s_dev, v_dev, nsrc, rad, part, st)));
  const size_t zsmem = (size_t)n_mom * 16 * sizeof(double2) + (size_t)nx * lz * sizeof(double2);
  TSM_CUDA(cudaFuncSetAttribute(project_z_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zsmem));
  count_launches(1);
  project_z_kernel<<<dim3(lt, 10), Z_BS, zsmem, st>>>(part, mom_dev, n_mom, lz, lt, rad, nx, 2.0 * kappa * mu,
                                                      out_dev, accumulate);
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

}  // namespace tsm
