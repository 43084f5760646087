// Twisted-mass Wilson stencil (Eq. 1's M and relatives) with a pluggable
// per-site epilogue and a deterministic per-right-hand-side reduction.
//
//   out(x) = in(x) + i tw g5 in(x)
//            - kappa sum_mu [ (1 + SF g_mu) U_mu(x) in(x+mu) + (1 - SF g_mu) U_mu(x-mu)^dag in(x-mu) ]
//
// SF = -1 gives M (tw = mu') and A (tw = 0); SF = +1 gives M^dag (tw = -mu').
// Gamma matrices are those of include/tsm.h (chiral basis): each
// (1 +- g_mu) has rank two, so the neighbour spinor is first projected onto a
// two-spin vector h, the colour matrix acts on h only, and the lower two
// spins are rebuilt from the upper ones.
//
// Thread mapping: one thread per (site, right-hand side).  The block index
// runs over (site tile, right-hand side) with the right-hand side fastest, so
// the blocks of all right-hand sides of one site tile are scheduled back to
// back and re-read that tile's links from L2 rather than from HBM.
//
// FP32 arithmetic (FP32, FP16 and BF16 fields) runs the colour products and
// accumulations in packed pairs (two-wide FP32 FMA) with the two projected
// spins side by side; FP64 and float-float sums use the scalar forms.
#pragma once

#include <type_traits>
#include <utility>

#include "common.cuh"

namespace tsm {

constexpr int DSLASH_BS = 128;

// Resident blocks per SM the register allocation must allow (__launch_bounds__),
// per field precision, as measured at 24^3 x 48: FP32 and 16-bit fields 7
// (<= 72 registers; 6 was 2.5% slower on the whole TSM step, 8 spills),
// float-float 3 (<= 168); FP64 keeps the compiler's choice.
// TSM_DSLASH_MINB32 / _MINB16 / _MINBDS override them (variant builds).
#ifndef TSM_DSLASH_MINB32
#define TSM_DSLASH_MINB32 7
#endif
#ifndef TSM_DSLASH_MINB16
#define TSM_DSLASH_MINB16 7
#endif
#ifndef TSM_DSLASH_MINBDS
#define TSM_DSLASH_MINBDS 3
#endif
template <int PIN>
struct MinBlocks {
  static constexpr int value =
      (PIN == TSM_F32) ? TSM_DSLASH_MINB32
                       : ((PIN == TSM_F16 || PIN == TSM_BF16) ? TSM_DSLASH_MINB16
                                                               : (PIN == TSM_DS ? TSM_DSLASH_MINBDS : 1));
};

struct DslashArgs {
  Geom g;
  const void* links;  // device links in the kernel's link precision
  const void* in;     // input field(s), native layout
  int nblk;           // blocks along the site axis
  int nrhs;           // right-hand sides in the launch
  double kappa;
  double tw;          // twist coefficient multiplying i g5
  float kappa_f, tw_f;  // the same, pre-rounded for FP32 kernels (no per-thread FP64 conversion)
  dsf kappa_ds, tw_ds;  // and split into float pairs for float-float kernels
  // checkerboarded operator (even-odd kernels only):
  //   out(j) = (c0 + i c1 g5) center(j) + (h0 + i h1 g5) hop(in)(j)
  // on the sites of parity `parity`, j = full site >> 1; center may be null.
  const void* center = nullptr;
  int parity = 0;
  double c0 = 0, c1 = 0, h0 = 0, h1 = 0;
  float c0_f = 0, c1_f = 0, h0_f = 0, h1_f = 0;
  dsf c0_ds{0.0f, 0.0f}, c1_ds{0.0f, 0.0f}, h0_ds{0.0f, 0.0f}, h1_ds{0.0f, 0.0f};
  // full-volume kernels: general = 1 replaces M by the coefficient form above
  int general = 0;
};

__host__ __device__ inline void set_eo(DslashArgs& a, const void* center, int parity, double c0, double c1, double h0,
                                       double h1) {
  a.center = center;
  a.parity = parity;
  a.c0 = c0;
  a.c1 = c1;
  a.h0 = h0;
  a.h1 = h1;
  a.c0_f = (float)c0;
  a.c1_f = (float)c1;
  a.h0_f = (float)h0;
  a.h1_f = (float)h1;
  a.c0_ds = dsf(c0);
  a.c1_ds = dsf(c1);
  a.h0_ds = dsf(h0);
  a.h1_ds = dsf(h1);
}

template <typename R>
struct EoCoef;
template <>
struct EoCoef<float> {
  __device__ static void get(const DslashArgs& a, float& c0, float& c1, float& h0, float& h1) {
    c0 = a.c0_f;
    c1 = a.c1_f;
    h0 = a.h0_f;
    h1 = a.h1_f;
  }
};
template <>
struct EoCoef<dsf> {
  __device__ static void get(const DslashArgs& a, dsf& c0, dsf& c1, dsf& h0, dsf& h1) {
    c0 = a.c0_ds;
    c1 = a.c1_ds;
    h0 = a.h0_ds;
    h1 = a.h1_ds;
  }
};
template <>
struct EoCoef<double> {
  __device__ static void get(const DslashArgs& a, double& c0, double& c1, double& h0, double& h1) {
    c0 = a.c0;
    c1 = a.c1;
    h0 = a.h0;
    h1 = a.h1;
  }
};

template <typename R>
__device__ __forceinline__ R arg_kappa(const DslashArgs& a);
template <>
__device__ __forceinline__ float arg_kappa<float>(const DslashArgs& a) { return a.kappa_f; }
template <>
__device__ __forceinline__ double arg_kappa<double>(const DslashArgs& a) { return a.kappa; }
template <>
__device__ __forceinline__ dsf arg_kappa<dsf>(const DslashArgs& a) { return a.kappa_ds; }
template <typename R>
__device__ __forceinline__ R arg_tw(const DslashArgs& a);
template <>
__device__ __forceinline__ float arg_tw<float>(const DslashArgs& a) { return a.tw_f; }
template <>
__device__ __forceinline__ double arg_tw<double>(const DslashArgs& a) { return a.tw; }
template <>
__device__ __forceinline__ dsf arg_tw<dsf>(const DslashArgs& a) { return a.tw_ds; }

__host__ __device__ inline void set_coeffs(DslashArgs& a, double kappa, double tw) {
  a.kappa = kappa;
  a.tw = tw;
  a.kappa_f = (float)kappa;
  a.tw_f = (float)tw;
  a.kappa_ds = dsf(kappa);
  a.tw_ds = dsf(tw);
}

struct RedSlots {
  double* partial;    // [nrhs][nblk]
  unsigned* counter;  // [nrhs], zero between launches
};

// ---------------------------------------------------------------- projection
// h = (upper two spins of) (1 + S g_MU) psi for the chiral basis:
//   MU = x: h0 = p0 - S i p3, h1 = p1 - S i p2      (i s1 = [[0, i], [i, 0]])
//   MU = y: h0 = p0 - S p3,   h1 = p1 + S p2        (i s2 = [[0, 1], [-1, 0]])
//   MU = z: h0 = p0 - S i p2, h1 = p1 + S i p3      (i s3 = diag(i, -i))
//   MU = t: h0 = p0 + S p2,   h1 = p1 + S p3
template <int MU, int S, typename T, class Add, class Sub, class MulI>
__device__ __forceinline__ void project_pair(T& h0, T& h1, T p0, T p1, T p2, T p3, Add add, Sub sub, MulI muli) {
  if (MU == 0) {
    h0 = S > 0 ? sub(p0, muli(p3)) : add(p0, muli(p3));
    h1 = S > 0 ? sub(p1, muli(p2)) : add(p1, muli(p2));
  } else if (MU == 1) {
    h0 = S > 0 ? sub(p0, p3) : add(p0, p3);
    h1 = S > 0 ? add(p1, p2) : sub(p1, p2);
  } else if (MU == 2) {
    h0 = S > 0 ? sub(p0, muli(p2)) : add(p0, muli(p2));
    h1 = S > 0 ? add(p1, muli(p3)) : sub(p1, muli(p3));
  } else {
    h0 = S > 0 ? add(p0, p2) : sub(p0, p2);
    h1 = S > 0 ? add(p1, p3) : sub(p1, p3);
  }
}

// Load the neighbour spinor of field r at site n and project it: h0, h1 (3 colours each).
template <int MU, int S, int PIN, typename R>
struct ProjLoad {
  __device__ __forceinline__ static void run(cplx<R> (&h0)[3], cplx<R> (&h1)[3], const void* base, size_t V, int r,
                                             int n) {
    cplx<R> p[12];
    SpinorIO<PIN>::load(base, V, r, n, p);
    auto add = [](cplx<R> a, cplx<R> b) { return a + b; };
    auto sub = [](cplx<R> a, cplx<R> b) { return a - b; };
    auto muli = [](cplx<R> a) { return times_i(a); };
#pragma unroll
    for (int c = 0; c < 3; ++c) project_pair<MU, S>(h0[c], h1[c], p[c], p[3 + c], p[6 + c], p[9 + c], add, sub, muli);
  }
};

// 16-bit storage: project in packed half2 / bfloat162 arithmetic, widen only h.
template <bool BF>
struct Packed2 {
  __device__ __forceinline__ static uint32_t add(uint32_t a, uint32_t b) {
    if (BF) {
      __nv_bfloat162 r = __hadd2(*reinterpret_cast<__nv_bfloat162*>(&a), *reinterpret_cast<__nv_bfloat162*>(&b));
      return *reinterpret_cast<uint32_t*>(&r);
    } else {
      __half2 r = __hadd2(*reinterpret_cast<__half2*>(&a), *reinterpret_cast<__half2*>(&b));
      return *reinterpret_cast<uint32_t*>(&r);
    }
  }
  __device__ __forceinline__ static uint32_t sub(uint32_t a, uint32_t b) {
    if (BF) {
      __nv_bfloat162 r = __hsub2(*reinterpret_cast<__nv_bfloat162*>(&a), *reinterpret_cast<__nv_bfloat162*>(&b));
      return *reinterpret_cast<uint32_t*>(&r);
    } else {
      __half2 r = __hsub2(*reinterpret_cast<__half2*>(&a), *reinterpret_cast<__half2*>(&b));
      return *reinterpret_cast<uint32_t*>(&r);
    }
  }
  // i (re, im) = (-im, re): swap the halves, flip the sign bit of the new real part
  __device__ __forceinline__ static uint32_t muli(uint32_t a) { return __byte_perm(a, 0, 0x1032) ^ 0x00008000u; }
  __device__ __forceinline__ static float2 widen(uint32_t w) { return BF ? b2f(w) : h2f(w); }
};

template <int MU, int S, bool BF, typename R>
__device__ __forceinline__ void proj_load_16(cplx<R> (&h0)[3], cplx<R> (&h1)[3], const void* base, size_t V, int r,
                                             int n) {
  const uint4* p = reinterpret_cast<const uint4*>(base) + (size_t)r * 3 * V + n;
  const uint4 a = __ldg(p), b = __ldg(p + V), c = __ldg(p + 2 * V);
  const uint32_t w[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
  using P2 = Packed2<BF>;
  auto add = [](uint32_t x, uint32_t y) { return P2::add(x, y); };
  auto sub = [](uint32_t x, uint32_t y) { return P2::sub(x, y); };
  auto muli = [](uint32_t x) { return P2::muli(x); };
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    uint32_t q0, q1;
    project_pair<MU, S>(q0, q1, w[col], w[3 + col], w[6 + col], w[9 + col], add, sub, muli);
    const float2 f0 = P2::widen(q0), f1 = P2::widen(q1);
    h0[col] = mk<R>(f0.x, f0.y);
    h1[col] = mk<R>(f1.x, f1.y);
  }
}
template <int MU, int S, typename R>
struct ProjLoad<MU, S, TSM_F16, R> {
  __device__ __forceinline__ static void run(cplx<R> (&h0)[3], cplx<R> (&h1)[3], const void* base, size_t V, int r,
                                             int n) {
    proj_load_16<MU, S, false, R>(h0, h1, base, V, r, n);
  }
};
template <int MU, int S, typename R>
struct ProjLoad<MU, S, TSM_BF16, R> {
  __device__ __forceinline__ static void run(cplx<R> (&h0)[3], cplx<R> (&h1)[3], const void* base, size_t V, int r,
                                             int n) {
    proj_load_16<MU, S, true, R>(h0, h1, base, V, r, n);
  }
};

// acc += (1 + S g_MU) W psi given h: w = W h (W = U, or U^dag when DAG), lower spins rebuilt.
template <int MU, int S, bool DAG, typename R>
__device__ __forceinline__ void hop_accumulate(cplx<R> (&acc)[12], const cplx<R> (&h0)[3], const cplx<R> (&h1)[3],
                                               const cplx<R> (&u)[3][3], R sgn) {
  const R s = (R)S;
  cplx<R> w0[3], w1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    w0[a] = mk<R>(0, 0);
    w1[a] = mk<R>(0, 0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (DAG) {
        cmacc(w0[a], u[b][a], h0[b]);
        cmacc(w1[a], u[b][a], h1[b]);
      } else {
        cmac(w0[a], u[a][b], h0[b]);
        cmac(w1[a], u[a][b], h1[b]);
      }
    }
    if (MU == 3) {  // only the time direction crosses the boundary
      w0[a] = sgn * w0[a];
      w1[a] = sgn * w1[a];
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc[a] = acc[a] + w0[a];
    acc[3 + a] = acc[3 + a] + w1[a];
    if (MU == 0) {          // lower = S i s1 w
      acc[6 + a] = acc[6 + a] + s * times_i(w1[a]);
      acc[9 + a] = acc[9 + a] + s * times_i(w0[a]);
    } else if (MU == 1) {
      acc[6 + a] = acc[6 + a] + s * w1[a];
      acc[9 + a] = acc[9 + a] - s * w0[a];
    } else if (MU == 2) {
      acc[6 + a] = acc[6 + a] + s * times_i(w0[a]);
      acc[9 + a] = acc[9 + a] - s * times_i(w1[a]);
    } else {                // lower = S w
      acc[6 + a] = acc[6 + a] + s * w0[a];
      acc[9 + a] = acc[9 + a] + s * w1[a];
    }
  }
}

// Both hops of direction MU for NR right-hand sides r0 .. r0+NR-1 (slots with
// act[j] false are skipped); each link is loaded and rebuilt once.
// Checkerboarded fields (EO = true) hold one parity at index i >> 1 with
// stride V / 2; links are always indexed by the full site.
template <int MU, int SF, typename R, int PIN, int PL, int NR, bool EO = false>
__device__ __forceinline__ void stencil_dir(cplx<R> (&acc)[NR][12], const DslashArgs& a, int r0,
                                            const bool (&act)[NR], int i, const int c[4]) {
  const size_t V = (size_t)a.g.V;
  const size_t FS = EO ? V / 2 : V;
  const int stride = dir_stride(a.g, MU);
  cplx<R> u[3][3];
  cplx<R> h0[3], h1[3];
  {  // forward: (1 + SF g) U_mu(x) psi(x + mu)
    const int n = fwd_site(a.g, i, c, MU, stride);
    LinkIO<PL>::load(a.links, V, MU, i, u);
    const R sgn = (MU == 3 && c[3] == a.g.L[3] - 1) ? (R)a.g.bc : (R)1;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (!act[j]) continue;
      ProjLoad<MU, SF, PIN, R>::run(h0, h1, a.in, FS, r0 + j, EO ? (n >> 1) : n);
      hop_accumulate<MU, SF, false>(acc[j], h0, h1, u, sgn);
    }
  }
  {  // backward: (1 - SF g) U_mu(x - mu)^dag psi(x - mu)
    const int n = bwd_site(a.g, i, c, MU, stride);
    LinkIO<PL>::load(a.links, V, MU, n, u);
    const R sgn = (MU == 3 && c[3] == 0) ? (R)a.g.bc : (R)1;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (!act[j]) continue;
      ProjLoad<MU, -SF, PIN, R>::run(h0, h1, a.in, FS, r0 + j, EO ? (n >> 1) : n);
      hop_accumulate<MU, -SF, true>(acc[j], h0, h1, u, sgn);
    }
  }
}

// f z for a unit factor f = sgn * (rot ? i : 1) (exact in every real type)
template <typename R>
__device__ __forceinline__ cplx<R> unit_times(cplx<R> z, bool rot, bool neg) {
  cplx<R> t = rot ? mk<R>(-z.im, z.re) : z;
  return neg ? mk<R>(-t.re, -t.im) : t;
}

// All eight hops of one site in a loop with the direction as a runtime value:
// one body instead of eight unrolled ones.  Used for float-float sums, whose
// unrolled form is too large for the instruction cache.  Same arithmetic as
// stencil_dir: h0 = p0 + f0 p_j0, h1 = p1 + f1 p_j1 (see project_pair),
// w = U h (U^dag on backward hops), lower spins = g0 w_k0, g1 w_k1.
template <int SF, typename R, int PIN, int PL, int NR, bool EO>
__device__ __forceinline__ void stencil_rolled(cplx<R> (&acc)[NR][12], const DslashArgs& a, int r0,
                                               const bool (&act)[NR], int i, const int c[4]) {
  const size_t V = (size_t)a.g.V;
  const size_t FS = EO ? V / 2 : V;
#pragma unroll 1
  for (int hop = 0; hop < 8; ++hop) {
    const int mu = hop >> 1;
    const bool back = (hop & 1) != 0;
    const int S = back ? -SF : SF;  // projector sign of this hop
    const int n = back ? bwd_site_rt(a.g, i, c, mu) : fwd_site_rt(a.g, i, c, mu);
    cplx<R> u[3][3];
    LinkIO<PL>::load(a.links, V, mu, back ? n : i, u);
    if (back) {  // U^dag in place
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        u[x][x] = conjc(u[x][x]);
#pragma unroll
        for (int y = x + 1; y < 3; ++y) {
          const cplx<R> t = u[x][y];
          u[x][y] = conjc(u[y][x]);
          u[y][x] = conjc(t);
        }
      }
    }
    const bool edge = (mu == 3) && (back ? (c[3] == 0) : (c[3] == a.g.L[3] - 1));
    const bool flip = edge && a.g.bc < 0;
    // projection h0 = p0 + f0 p_j0, h1 = p1 + f1 p_j1
    const int j0 = (mu == 0 || mu == 1) ? 3 : 2, j1 = 5 - j0;
    const bool rot = (mu == 0 || mu == 2);
    const bool neg0 = (mu == 3) ? (S < 0) : (S > 0);
    const bool neg1 = (mu == 0) ? (S > 0) : (S < 0);
    // lower spins: acc6 += g0 w_k0, acc9 += g1 w_k1
    const int k0 = (mu == 0 || mu == 1) ? 1 : 0;
    const bool gneg0 = (S < 0);
    const bool gneg1 = (mu == 1 || mu == 2) ? (S > 0) : (S < 0);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      if (!act[q]) continue;
      cplx<R> p[12];
      SpinorIO<PIN>::load(a.in, FS, r0 + q, EO ? (n >> 1) : n, p);
      cplx<R> h0[3], h1[3];
#pragma unroll
      for (int col = 0; col < 3; ++col) {  // spins j0, j1 selected, not indexed (p stays in registers)
        const cplx<R> pj0 = j0 == 3 ? p[9 + col] : p[6 + col], pj1 = j1 == 3 ? p[9 + col] : p[6 + col];
        h0[col] = p[col] + unit_times(pj0, rot, neg0);
        h1[col] = p[3 + col] + unit_times(pj1, rot, neg1);
      }
      cplx<R> w0[3], w1[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        w0[x] = mk<R>(0, 0);
        w1[x] = mk<R>(0, 0);
#pragma unroll
        for (int y = 0; y < 3; ++y) {
          cmac(w0[x], u[x][y], h0[y]);
          cmac(w1[x], u[x][y], h1[y]);
        }
        if (flip) {
          w0[x] = mk<R>(-w0[x].re, -w0[x].im);
          w1[x] = mk<R>(-w1[x].re, -w1[x].im);
        }
      }
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        acc[q][x] = acc[q][x] + w0[x];
        acc[q][3 + x] = acc[q][3 + x] + w1[x];
        const cplx<R> a0 = k0 ? w1[x] : w0[x], a1 = k0 ? w0[x] : w1[x];
        acc[q][6 + x] = acc[q][6 + x] + unit_times(a0, rot, gneg0);
        acc[q][9 + x] = acc[q][9 + x] + unit_times(a1, rot, gneg1);
      }
    }
  }
}

// One hop in packed-pair arithmetic (Blackwell's two-wide FP32 FMA,
// __ffma2_rn): the two projected spins travel together as pairs
// hr[b] = (h0[b].re, h1[b].re), hi[b] = (h0[b].im, h1[b].im), so that one
// two-wide FMA serves both spins.  Results come back per spin pair:
// up[0..2] = (spin 0, spin 1) real parts, up[3..5] imaginary parts, and lo[]
// likewise for spins (2, 3), except that for MU = x, y (whose lower spins
// take the other upper spin) lo holds (spin 3, spin 2).
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }

template <int MU, int S, bool DAG, bool FIRST>
__device__ __forceinline__ void hop_pairs(float2 (&up)[6], float2 (&lo)[6], const cplx<float> (&h0)[3],
                                          const cplx<float> (&h1)[3], const cplx<float> (&u)[3][3], float sgn) {
  float2 hr[3], hi[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    hr[b] = make_float2(h0[b].re, h1[b].re);
    hi[b] = make_float2(h0[b].im, h1[b].im);
  }
  float2 wr[3], wi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // W = U (or U^dag): w = W h;  W_ab = (ur, ui)
      const float ur = DAG ? u[b][a].re : u[a][b].re;
      const float ui = DAG ? -u[b][a].im : u[a][b].im;
      if (b == 0) {
        wr[a] = __fmul2_rn(bcast2(ur), hr[0]);
        wi[a] = __fmul2_rn(bcast2(ur), hi[0]);
      } else {
        wr[a] = __ffma2_rn(bcast2(ur), hr[b], wr[a]);
        wi[a] = __ffma2_rn(bcast2(ur), hi[b], wi[a]);
      }
      wr[a] = __ffma2_rn(bcast2(-ui), hi[b], wr[a]);
      wi[a] = __ffma2_rn(bcast2(ui), hr[b], wi[a]);
    }
  }
  // upper spins: + sgn w;  lower spins per projector (see hop_accumulate)
  const float s = (float)S * sgn;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (FIRST) {
      up[a] = __fmul2_rn(bcast2(sgn), wr[a]);
      up[3 + a] = __fmul2_rn(bcast2(sgn), wi[a]);
    } else {
      up[a] = __ffma2_rn(bcast2(sgn), wr[a], up[a]);
      up[3 + a] = __ffma2_rn(bcast2(sgn), wi[a], up[3 + a]);
    }
    float2 cr, ci, vr, vi;  // lo += cr * vr (real pair), ci * vi (imaginary pair)
    if (MU == 0) {          // (s3, s2) += S i (w0, w1)
      cr = bcast2(-s); vr = wi[a];
      ci = bcast2(s);  vi = wr[a];
    } else if (MU == 1) {   // (s3, s2) += S (-w0, w1)
      cr = make_float2(-s, s); vr = wr[a];
      ci = make_float2(-s, s); vi = wi[a];
    } else if (MU == 2) {   // (s2, s3) += S i (w0, -w1)
      cr = make_float2(-s, s); vr = wi[a];
      ci = make_float2(s, -s); vi = wr[a];
    } else {                // (s2, s3) += S sgn (w0, w1)
      cr = bcast2(s); vr = wr[a];
      ci = bcast2(s); vi = wi[a];
    }
    if (FIRST) {
      lo[a] = __fmul2_rn(cr, vr);
      lo[3 + a] = __fmul2_rn(ci, vi);
    } else {
      lo[a] = __ffma2_rn(cr, vr, lo[a]);
      lo[3 + a] = __ffma2_rn(ci, vi, lo[3 + a]);
    }
  }
}

// Both hops of direction MU for NR right-hand sides in packed pairs (each
// link loaded and rebuilt once); FIRST initialises the accumulators.
template <int MU, int SF, int PIN, int PL, int NR, bool EO, bool FIRST>
__device__ __forceinline__ void pairs_dir(float2 (&up)[NR][6], float2 (&lo)[NR][6], const DslashArgs& a, int r0,
                                          const bool (&act)[NR], int i, const int c[4]) {
  const size_t V = (size_t)a.g.V;
  const size_t FS = EO ? V / 2 : V;
  const int stride = dir_stride(a.g, MU);
  cplx<float> u[3][3], h0[3], h1[3];
  {
    const int n = fwd_site(a.g, i, c, MU, stride);
    LinkIO<PL>::load(a.links, V, MU, i, u);
    const float sgn = (MU == 3 && c[3] == a.g.L[3] - 1) ? (float)a.g.bc : 1.0f;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (!act[j]) {  // inactive slots are never read; FIRST still defines them
        if (FIRST) {
#pragma unroll
          for (int k = 0; k < 6; ++k) up[j][k] = lo[j][k] = make_float2(0.0f, 0.0f);
        }
        continue;
      }
      ProjLoad<MU, SF, PIN, float>::run(h0, h1, a.in, FS, r0 + j, EO ? (n >> 1) : n);
      hop_pairs<MU, SF, false, FIRST>(up[j], lo[j], h0, h1, u, sgn);
    }
  }
  {
    const int n = bwd_site(a.g, i, c, MU, stride);
    LinkIO<PL>::load(a.links, V, MU, n, u);
    const float sgn = (MU == 3 && c[3] == 0) ? (float)a.g.bc : 1.0f;
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (!act[j]) continue;
      ProjLoad<MU, -SF, PIN, float>::run(h0, h1, a.in, FS, r0 + j, EO ? (n >> 1) : n);
      hop_pairs<MU, -SF, true, false>(up[j], lo[j], h0, h1, u, sgn);
    }
  }
}

// All eight hops of one site in packed pairs, for NR right-hand sides; out
// receives the hop sum in component order.  Directions x and y leave the
// lower spins in (3, 2) order; one swap before z restores (2, 3).
template <int SF, int PIN, int PL, int NR, bool EO>
__device__ __forceinline__ void stencil_pairs(cplx<float> (&out)[NR][12], const DslashArgs& a, int r0,
                                              const bool (&act)[NR], int i, const int c[4]) {
  float2 up[NR][6], lo[NR][6];
  pairs_dir<0, SF, PIN, PL, NR, EO, true>(up, lo, a, r0, act, i, c);
  pairs_dir<1, SF, PIN, PL, NR, EO, false>(up, lo, a, r0, act, i, c);
#pragma unroll
  for (int j = 0; j < NR; ++j)
#pragma unroll
    for (int k = 0; k < 6; ++k) lo[j][k] = make_float2(lo[j][k].y, lo[j][k].x);
  pairs_dir<2, SF, PIN, PL, NR, EO, false>(up, lo, a, r0, act, i, c);
  pairs_dir<3, SF, PIN, PL, NR, EO, false>(up, lo, a, r0, act, i, c);
#pragma unroll
  for (int j = 0; j < NR; ++j)
#pragma unroll
    for (int col = 0; col < 3; ++col) {
      out[j][col] = mk<float>(up[j][col].x, up[j][3 + col].x);
      out[j][3 + col] = mk<float>(up[j][col].y, up[j][3 + col].y);
      out[j][6 + col] = mk<float>(lo[j][col].x, lo[j][3 + col].x);
      out[j][9 + col] = mk<float>(lo[j][col].y, lo[j][3 + col].y);
    }
}

// Full operator at site i for NR right-hand sides: out = in + i tw g5 in - kappa * hop.
template <int SF, typename R, int PIN, int PL, int NR, bool P2 = std::is_same<R, float>::value>
__device__ __forceinline__ void apply_site(cplx<R> (&out)[NR][12], const DslashArgs& a, int r0, const bool (&act)[NR],
                                           int i) {
  int c[4];
  site_coords(a.g, i, c);
  if constexpr (P2 && std::is_same<R, float>::value) {
    stencil_pairs<SF, PIN, PL, NR, false>(out, a, r0, act, i, c);
  } else {
#pragma unroll
    for (int j = 0; j < NR; ++j)
#pragma unroll
      for (int k = 0; k < 12; ++k) out[j][k] = mk<R>(0, 0);
  }
  if constexpr (P2 && std::is_same<R, float>::value) {
    // done above
  } else if constexpr (std::is_same<R, dsf>::value) {
    stencil_rolled<SF, R, PIN, PL, NR, false>(out, a, r0, act, i, c);
  } else {
    stencil_dir<0, SF, R, PIN, PL, NR>(out, a, r0, act, i, c);
    stencil_dir<1, SF, R, PIN, PL, NR>(out, a, r0, act, i, c);
    stencil_dir<2, SF, R, PIN, PL, NR>(out, a, r0, act, i, c);
    stencil_dir<3, SF, R, PIN, PL, NR>(out, a, r0, act, i, c);
  }
  if (a.general) {  // (c0 + i c1 g5) centre + (h0 + i h1 g5) hop
    R c0, c1, h0, h1;
    EoCoef<R>::get(a, c0, c1, h0, h1);
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (!act[j]) continue;
      cplx<R> ctr[12];
      if (a.center) {
        SpinorIO<PIN>::load(a.center, (size_t)a.g.V, r0 + j, i, ctr);
      } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) ctr[k] = mk<R>(0, 0);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const R g5 = (k < 6) ? (R)1 : (R)-1;
        const cplx<R> hv = out[j][k];
        out[j][k] = c0 * ctr[k] + (g5 * c1) * times_i(ctr[k]) + h0 * hv + (g5 * h1) * times_i(hv);
      }
    }
    return;
  }
  const R kap = arg_kappa<R>(a), tw = arg_tw<R>(a);
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    if (!act[j]) continue;
    cplx<R> ctr[12];
    SpinorIO<PIN>::load(a.in, (size_t)a.g.V, r0 + j, i, ctr);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R g5 = (k < 6) ? (R)1 : (R)-1;
      cplx<R> t = ctr[k] + (g5 * tw) * times_i(ctr[k]);
      out[j][k] = t - kap * out[j][k];
    }
  }
}

// Last-block-done reduction: every block adds its partial to slot
// [rhs][block]; the block that arrives last sums the slots in fixed order
// (deterministic for a fixed grid) and calls epi.finalize(rhs, total).
template <class Epi>
__device__ __forceinline__ void reduce_and_finalize(const Epi& epi, const RedSlots& red, int rhs, int nblk,
                                                    int blk, double v, double* sh) {
  __shared__ bool is_last;
  double bs = block_sum(v, sh);
  if (threadIdx.x == 0) {
    red.partial[(size_t)rhs * nblk + blk] = bs;
    __threadfence();
    unsigned t = atomicAdd(&red.counter[rhs], 1u);
    is_last = (t == (unsigned)(nblk - 1));
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double s = 0.0;
    for (int j = threadIdx.x; j < nblk; j += blockDim.x) s += __ldcg(&red.partial[(size_t)rhs * nblk + j]);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      epi.finalize(rhs, s);
      red.counter[rhs] = 0;
    }
  }
}

// Epilogue interface:
//   static constexpr bool kReduce;
//   bool active(int rhs)                      -- block-uniform skip
//   R site(int rhs, int i, cplx<R>(&out)[12]) -- consume the result, return the value to sum
//   void finalize(int rhs, double total)      -- last block, thread 0
//   RedSlots red;
// One block of work: bid = site_block * ngroups + group, group = NR
// consecutive right-hand sides.  Shared by the single-instance kernel below
// and the multi-instance kernels of the batched solver.
template <typename R, int SF, int PIN, int PL, int NR, class Epi, bool P2 = std::is_same<R, float>::value>
__device__ __forceinline__ void dslash_block(const DslashArgs& a, const Epi& epi, int bid) {
  __shared__ double sh[32];
  const int ngrp = (a.nrhs + NR - 1) / NR;
  const int grp = bid % ngrp;
  const int blk = bid / ngrp;
  const int r0 = grp * NR;
  bool act[NR];
  bool any = false;
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    act[j] = (r0 + j < a.nrhs) && epi.active(r0 + j);
    any |= act[j];
  }
  if (!any) return;
  const int i = blk * DSLASH_BS + threadIdx.x;
  R red[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) red[j] = (R)0;
  if (i < a.g.V) {
    cplx<R> out[NR][12];
    apply_site<SF, R, PIN, PL, NR, P2>(out, a, r0, act, i);
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (act[j]) red[j] = epi.site(r0 + j, i, out[j]);
  }
  if (Epi::kReduce) {
#pragma unroll
    for (int j = 0; j < NR; ++j)
      if (act[j]) reduce_and_finalize(epi, epi.red, r0 + j, a.nblk, blk, (double)red[j], sh);
  }
}

template <typename R, int SF, int PIN, int PL, int NR, class Epi, bool P2 = std::is_same<R, float>::value>
__global__ void __launch_bounds__(DSLASH_BS, MinBlocks<PIN>::value) dslash_kernel(DslashArgs a, Epi epi) {
  dslash_block<R, SF, PIN, PL, NR, Epi, P2>(a, epi, blockIdx.x);
}

// ---------------------------------------------------------------- even-odd operator
// Full site of checkerboard index j on parity p (all extents even: sites 2j
// and 2j+1 share y, z, t and have opposite parity).
__device__ __forceinline__ int eo_site(const Geom& g, int j, int p, int c[4]) {
  const int i0 = 2 * j;
  site_coords(g, i0, c);
  const int b = (p - (c[1] + c[2] + c[3])) & 1;  // x of i0 is even
  c[0] += b;
  return i0 + b;
}

template <int SF, typename R, int PIN, int PL, int NR, bool P2 = std::is_same<R, float>::value>
__device__ __forceinline__ void apply_site_eo(cplx<R> (&out)[NR][12], const DslashArgs& a, int r0,
                                              const bool (&act)[NR], int j) {
  int c[4];
  const int i = eo_site(a.g, j, a.parity, c);
  if constexpr (P2 && std::is_same<R, float>::value) {
    stencil_pairs<SF, PIN, PL, NR, true>(out, a, r0, act, i, c);
  } else {
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int k = 0; k < 12; ++k) out[q][k] = mk<R>(0, 0);
  }
  if constexpr (P2 && std::is_same<R, float>::value) {
    // done above
  } else if constexpr (std::is_same<R, dsf>::value) {
    stencil_rolled<SF, R, PIN, PL, NR, true>(out, a, r0, act, i, c);
  } else {
    stencil_dir<0, SF, R, PIN, PL, NR, true>(out, a, r0, act, i, c);
    stencil_dir<1, SF, R, PIN, PL, NR, true>(out, a, r0, act, i, c);
    stencil_dir<2, SF, R, PIN, PL, NR, true>(out, a, r0, act, i, c);
    stencil_dir<3, SF, R, PIN, PL, NR, true>(out, a, r0, act, i, c);
  }
  R c0, c1, h0, h1;
  EoCoef<R>::get(a, c0, c1, h0, h1);
  const size_t FS = (size_t)a.g.V / 2;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    if (!act[q]) continue;
    cplx<R> ctr[12];
    if (a.center) {
      SpinorIO<PIN>::load(a.center, FS, r0 + q, j, ctr);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) ctr[k] = mk<R>(0, 0);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R g5 = (k < 6) ? (R)1 : (R)-1;
      const cplx<R> hv = out[q][k];
      out[q][k] = c0 * ctr[k] + (g5 * c1) * times_i(ctr[k]) + h0 * hv + (g5 * h1) * times_i(hv);
    }
  }
}

template <typename R, int SF, int PIN, int PL, int NR, class Epi, bool P2 = std::is_same<R, float>::value>
__device__ __forceinline__ void dslash_block_eo(const DslashArgs& a, const Epi& epi, int bid) {
  __shared__ double sh[32];
  const int ngrp = (a.nrhs + NR - 1) / NR;
  const int grp = bid % ngrp;
  const int blk = bid / ngrp;
  const int r0 = grp * NR;
  bool act[NR];
  bool any = false;
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    act[q] = (r0 + q < a.nrhs) && epi.active(r0 + q);
    any |= act[q];
  }
  if (!any) return;
  const int j = blk * DSLASH_BS + threadIdx.x;
  R red[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) red[q] = (R)0;
  if (j < a.g.V / 2) {
    cplx<R> out[NR][12];
    apply_site_eo<SF, R, PIN, PL, NR, P2>(out, a, r0, act, j);
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (act[q]) red[q] = epi.site(r0 + q, j, out[q]);
  }
  if (Epi::kReduce) {
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (act[q]) reduce_and_finalize(epi, epi.red, r0 + q, a.nblk, blk, (double)red[q], sh);
  }
}

template <typename R, int SF, int PIN, int PL, int NR, class Epi, bool P2 = std::is_same<R, float>::value>
__global__ void __launch_bounds__(DSLASH_BS, MinBlocks<PIN>::value) dslash_eo_kernel(DslashArgs a, Epi epi) {
  dslash_block_eo<R, SF, PIN, PL, NR, Epi, P2>(a, epi, blockIdx.x);
}

// a.nblk must be ceil(V/2 / DSLASH_BS); nr right-hand sides per thread (1, 2
// or 4; 4 only for FP32 sums).
template <typename R, int SF, int PIN, int PL, class Epi>
inline void launch_dslash_eo(int nr, const DslashArgs& a, const Epi& e, cudaStream_t s) {
  const unsigned nb = (unsigned)a.nblk;
  if constexpr (sizeof(R) == 4) {
    if (nr == 4) {
      dslash_eo_kernel<R, SF, PIN, PL, 4, Epi><<<nb * (unsigned)((a.nrhs + 3) / 4), DSLASH_BS, 0, s>>>(a, e);
      return;
    }
  }
  if (nr >= 2) {
    dslash_eo_kernel<R, SF, PIN, PL, 2, Epi><<<nb * (unsigned)((a.nrhs + 1) / 2), DSLASH_BS, 0, s>>>(a, e);
  } else {
    dslash_eo_kernel<R, SF, PIN, PL, 1, Epi><<<nb * (unsigned)a.nrhs, DSLASH_BS, 0, s>>>(a, e);
  }
}

// Plain store of the result (optionally times g5), no reduction.
template <typename R, int PO>
struct EpiStore {
  static constexpr bool kReduce = false;
  void* out;
  size_t V;
  int gamma5;
  RedSlots red;
  __device__ bool active(int) const { return true; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    if (gamma5) {
#pragma unroll
      for (int k = 6; k < 12; ++k) o[k] = mk<R>(-o[k].re, -o[k].im);
    }
    SpinorIO<PO>::store(out, V, rhs, i, o);
    return (R)0;
  }
  __device__ void finalize(int, double) const {}
};

inline dim3 dslash_grid(int V, int nrhs, int nr) {
  return dim3((unsigned)((V + DSLASH_BS - 1) / DSLASH_BS) * (unsigned)((nrhs + nr - 1) / nr), 1, 1);
}

// Launch with nr right-hand sides per thread (1, 2 or 4; chosen by the autotuner).
template <typename R, int SF, int PIN, int PL, class Epi>
inline void launch_dslash(int nr, const DslashArgs& a, const Epi& e, cudaStream_t s) {
  if constexpr (sizeof(R) == 4) {
    if (nr == 4) {
      dslash_kernel<R, SF, PIN, PL, 4, Epi><<<dslash_grid(a.g.V, a.nrhs, 4), DSLASH_BS, 0, s>>>(a, e);
      return;
    }
  }
  // FP64 sums do not fit 4 right-hand sides in registers: at most 2 there
  if (nr >= 2) {
    dslash_kernel<R, SF, PIN, PL, 2, Epi><<<dslash_grid(a.g.V, a.nrhs, 2), DSLASH_BS, 0, s>>>(a, e);
  } else {
    dslash_kernel<R, SF, PIN, PL, 1, Epi><<<dslash_grid(a.g.V, a.nrhs, 1), DSLASH_BS, 0, s>>>(a, e);
  }
}

}  // namespace tsm
