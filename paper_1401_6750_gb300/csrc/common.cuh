// Device-side building blocks shared by the kernels of the library:
// complex arithmetic, the chunked spinor layout, compressed link storage and
// lattice geometry.  Conventions are those of include/tsm.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

#include "tsm.h"

namespace tsm {

// Internal storage precision of the precise operator of the reliable-update
// solver: each real as a pair of floats (hi + lo), 16 bytes per complex like
// TSM_F64.  Not part of the public precision enumeration.
constexpr int TSM_DS = 4;

// ---------------------------------------------------------------- float-float
// A real carried as an unevaluated sum hi + lo of two floats (about 44 bits
// of significand after a few dozen operations), so that the FP32 pipes do the
// work of an FP64 operator.  Sums use Knuth's TwoSum (TAOCP vol. 2, 4.2.2)
// for the leading parts and add the trailing parts with plain float adds;
// products use the FMA form of Dekker's exact product (Dekker 1971) plus the
// cross and lo * lo terms.  lo is left unnormalised between operations and
// renormalised (TwoSum) when stored.
struct dsf {
  float hi, lo;
  dsf() = default;
  __host__ __device__ __forceinline__ dsf(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ dsf(float v) : hi(v), lo(0.0f) {}
  __host__ __device__ __forceinline__ dsf(int v) : hi((float)v), lo(0.0f) {}
  __host__ __device__ __forceinline__ dsf(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return dsf(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf& operator+=(dsf& a, dsf b) { return a = a + b; }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }
// The lo * lo term stays: after a cancellation lo can exceed hi, and the
// square of such a value (a residual component) needs it.
__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  e = fmaf(a.lo, b.lo, e);
  return dsf(p, e);
}
// a * b + c for every real type of the kernels (exact-type overloads)
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ dsf fmar(dsf a, dsf b, dsf c) { return a * b + c; }
// hi = fl(hi + lo), lo = the rounding error (TwoSum: exact whatever the
// relative size of the parts)
__device__ __forceinline__ dsf normalise(dsf a) {
  const float s = a.hi + a.lo;
  const float bb = s - a.hi;
  return dsf(s, (a.hi - (s - bb)) + (a.lo - bb));
}

// Arithmetic of element-wise kernels over fields of precisions P...: double
// when any of them carries more than a float (FP64, float-float), float
// otherwise (GB300's FP64 pipe, conversions included, is 1/64 of FP32).
template <int... P>
struct EwReal {
  static constexpr bool wide = ((P == TSM_F64 || P == TSM_DS) || ...);
  using type = typename std::conditional<wide, double, float>::type;
};
template <int... P>
using ew_real = typename EwReal<P...>::type;

// ---------------------------------------------------------------- complex
template <typename R>
struct cplx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R re, R im) {
  cplx<R> c;
  c.re = re;
  c.im = im;
  return c;
}
template <typename R>
__device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R>
__device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R>
__device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R>
__device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// conj(a) * b
template <typename R>
__device__ __forceinline__ cplx<R> cmulc(cplx<R> a, cplx<R> b) {
  return mk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// acc += a * b
template <typename R>
__device__ __forceinline__ void cmac(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fmar(a.re, b.re, acc.re);
  acc.re = fmar(-a.im, b.im, acc.re);
  acc.im = fmar(a.re, b.im, acc.im);
  acc.im = fmar(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__device__ __forceinline__ void cmacc(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fmar(a.re, b.re, acc.re);
  acc.re = fmar(a.im, b.im, acc.re);
  acc.im = fmar(a.re, b.im, acc.im);
  acc.im = fmar(-a.im, b.re, acc.im);
}
template <typename R>
__device__ __forceinline__ cplx<R> times_i(cplx<R> a) { return mk(-a.im, a.re); }
template <typename R>
__device__ __forceinline__ cplx<R> conjc(cplx<R> a) { return mk(a.re, -a.im); }
template <typename R>
__device__ __forceinline__ R norm2(cplx<R> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------- geometry
// Exact unsigned division by an invariant d through multiply and shift
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, for every 32-bit n
//   t = mulhi(m, n),  n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
  uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__host__ __device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  const uint32_t t = __umulhi(f.m, n);
#else
  const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

struct Geom {
  int L[4];  // Lx, Ly, Lz, T
  int V;
  int bc;    // temporal boundary sign on the last timeslice
  FastDiv div[3];  // by Lx, Ly, Lz
};

__device__ __forceinline__ void site_coords(const Geom& g, int i, int c[4]) {
  uint32_t q = fast_div((uint32_t)i, g.div[0]);
  c[0] = i - (int)q * g.L[0];
  uint32_t q2 = fast_div(q, g.div[1]);
  c[1] = (int)q - (int)q2 * g.L[1];
  uint32_t q3 = fast_div(q2, g.div[2]);
  c[2] = (int)q2 - (int)q3 * g.L[2];
  c[3] = (int)q3;
}

// strides of the lexicographic site index
__device__ __forceinline__ int dir_stride(const Geom& g, int mu) {
  int s = 1;
  for (int m = 0; m < mu; ++m) s *= g.L[m];
  return s;
}

__device__ __forceinline__ int fwd_site(const Geom& g, int i, const int c[4], int mu, int stride) {
  return (c[mu] == g.L[mu] - 1) ? i - (g.L[mu] - 1) * stride : i + stride;
}
__device__ __forceinline__ int bwd_site(const Geom& g, int i, const int c[4], int mu, int stride) {
  return (c[mu] == 0) ? i + (g.L[mu] - 1) * stride : i - stride;
}
// Forward neighbour for a direction known only at run time, written with
// selects: an array or kernel-parameter field indexed at run time is copied
// to local memory by the compiler (a per-thread stack frame).
__device__ __forceinline__ int fwd_site_rt(const Geom& g, int i, const int c[4], int mu) {
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
  const int cm = mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
  const int lm = mu == 0 ? L0 : (mu == 1 ? L1 : (mu == 2 ? L2 : L3));
  const int st = mu == 0 ? 1 : (mu == 1 ? L0 : (mu == 2 ? L0 * L1 : L0 * L1 * L2));
  return cm == lm - 1 ? i - (lm - 1) * st : i + st;
}
__device__ __forceinline__ int bwd_site_rt(const Geom& g, int i, const int c[4], int mu) {
  const int L0 = g.L[0], L1 = g.L[1], L2 = g.L[2], L3 = g.L[3];
  const int cm = mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
  const int lm = mu == 0 ? L0 : (mu == 1 ? L1 : (mu == 2 ? L2 : L3));
  const int st = mu == 0 ? 1 : (mu == 1 ? L0 : (mu == 2 ? L0 * L1 : L0 * L1 * L2));
  return cm == 0 ? i + (lm - 1) * st : i - st;
}

// ---------------------------------------------------------------- spinor IO
// Chunked layout: chunk j of site i of field r at ((r*NCH + j)*V + i)*16 bytes.
template <int P>
struct SpinorIO;

template <>
struct SpinorIO<TSM_F64> {
  static constexpr int NCH = 12;
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int r, int i, cplx<R> (&v)[12]) {
    const double2* p = reinterpret_cast<const double2*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 d = __ldg(p + k * V);
      v[k] = mk<R>((R)d.x, (R)d.y);
    }
  }
  template <typename R>
  __device__ __forceinline__ static void store(void* base, size_t V, int r, int i, const cplx<R> (&v)[12]) {
    double2* p = reinterpret_cast<double2*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * V] = make_double2((double)v[k].re, (double)v[k].im);
  }
};

template <>
struct SpinorIO<TSM_F32> {
  static constexpr int NCH = 6;
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int r, int i, cplx<R> (&v)[12]) {
    const float4* p = reinterpret_cast<const float4*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      float4 d = __ldg(p + k * V);
      v[2 * k] = mk<R>((R)d.x, (R)d.y);
      v[2 * k + 1] = mk<R>((R)d.z, (R)d.w);
    }
  }
  template <typename R>
  __device__ __forceinline__ static void store(void* base, size_t V, int r, int i, const cplx<R> (&v)[12]) {
    float4* p = reinterpret_cast<float4*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 6; ++k)
      p[k * V] = make_float4((float)v[2 * k].re, (float)v[2 * k].im, (float)v[2 * k + 1].re,
                             (float)v[2 * k + 1].im);
  }
};

__device__ __forceinline__ float2 h2f(uint32_t w) { return __half22float2(*reinterpret_cast<__half2*>(&w)); }
__device__ __forceinline__ float2 b2f(uint32_t w) {
  return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w));
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t f2b(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

template <bool BF>
struct Half16IO {
  static constexpr int NCH = 3;
  __device__ __forceinline__ static float2 cvt(uint32_t w) { return BF ? b2f(w) : h2f(w); }
  __device__ __forceinline__ static uint32_t pack(float a, float b) { return BF ? f2b(a, b) : f2h(a, b); }
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int r, int i, cplx<R> (&v)[12]) {
    const uint4* p = reinterpret_cast<const uint4*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 d = __ldg(p + k * V);
      float2 a = cvt(d.x), b = cvt(d.y), c = cvt(d.z), e = cvt(d.w);
      v[4 * k] = mk<R>(a.x, a.y);
      v[4 * k + 1] = mk<R>(b.x, b.y);
      v[4 * k + 2] = mk<R>(c.x, c.y);
      v[4 * k + 3] = mk<R>(e.x, e.y);
    }
  }
  template <typename R>
  __device__ __forceinline__ static void store(void* base, size_t V, int r, int i, const cplx<R> (&v)[12]) {
    uint4* p = reinterpret_cast<uint4*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 d;
      d.x = pack((float)v[4 * k].re, (float)v[4 * k].im);
      d.y = pack((float)v[4 * k + 1].re, (float)v[4 * k + 1].im);
      d.z = pack((float)v[4 * k + 2].re, (float)v[4 * k + 2].im);
      d.w = pack((float)v[4 * k + 3].re, (float)v[4 * k + 3].im);
      p[k * V] = d;
    }
  }
};
template <>
struct SpinorIO<TSM_F16> : Half16IO<false> {};
template <>
struct SpinorIO<TSM_BF16> : Half16IO<true> {};

// float-float: one float4 (re.hi, re.lo, im.hi, im.lo) per complex, 12 chunks
template <typename R>
__device__ __forceinline__ R from_pair(float h, float l) {
  return (R)((double)h + (double)l);
}
template <>
__device__ __forceinline__ float from_pair<float>(float h, float l) { return h + l; }
template <>
__device__ __forceinline__ dsf from_pair<dsf>(float h, float l) { return dsf(h, l); }
template <typename R>
__device__ __forceinline__ dsf to_pair(R v) { return dsf((double)v); }
template <>
__device__ __forceinline__ dsf to_pair<float>(float v) { return dsf(v); }
template <>
__device__ __forceinline__ dsf to_pair<dsf>(dsf v) { return normalise(v); }

template <>
struct SpinorIO<TSM_DS> {
  static constexpr int NCH = 12;
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int r, int i, cplx<R> (&v)[12]) {
    const float4* p = reinterpret_cast<const float4*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float4 d = __ldg(p + k * V);
      v[k] = mk<R>(from_pair<R>(d.x, d.y), from_pair<R>(d.z, d.w));
    }
  }
  template <typename R>
  __device__ __forceinline__ static void store(void* base, size_t V, int r, int i, const cplx<R> (&v)[12]) {
    float4* p = reinterpret_cast<float4*>(base) + (size_t)r * NCH * V + i;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const dsf a = to_pair<R>(v[k].re), b = to_pair<R>(v[k].im);
      p[k * V] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
  }
};

__host__ __device__ constexpr int spinor_chunks(int p) {
  return (p == TSM_F64 || p == TSM_DS) ? 12 : (p == TSM_F32 ? 6 : 3);
}

// ---------------------------------------------------------------- links
// F64: [4][9][V] double2, all entries U_ab (k = 3a + b).
// F32: [4][3][V] float4, rows 0 and 1 (6 complex, row-major).
// F16/BF16: [4][V] uint4 (U00, U01, U02, U10) then [4][V] uint2 (U11, U12).
// Compressed forms rebuild row 2 = conj(row0 x row1).
template <typename R>
__device__ __forceinline__ void reconstruct_row2(cplx<R> (&u)[3][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    cplx<R> t = cmul(u[0][c1], u[1][c2]) - cmul(u[0][c2], u[1][c1]);
    u[2][c] = conjc(t);
  }
}

template <int P>
struct LinkIO;

template <>
struct LinkIO<TSM_F64> {
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int mu, int i, cplx<R> (&u)[3][3]) {
    const double2* p = reinterpret_cast<const double2*>(base) + (size_t)mu * 9 * V + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 d = __ldg(p + k * V);
      u[k / 3][k % 3] = mk<R>((R)d.x, (R)d.y);
    }
  }
};

template <>
struct LinkIO<TSM_F32> {
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int mu, int i, cplx<R> (&u)[3][3]) {
    const float4* p = reinterpret_cast<const float4*>(base) + (size_t)mu * 3 * V + i;
    float4 a = __ldg(p), b = __ldg(p + V), c = __ldg(p + 2 * V);
    u[0][0] = mk<R>(a.x, a.y);
    u[0][1] = mk<R>(a.z, a.w);
    u[0][2] = mk<R>(b.x, b.y);
    u[1][0] = mk<R>(b.z, b.w);
    u[1][1] = mk<R>(c.x, c.y);
    u[1][2] = mk<R>(c.z, c.w);
    reconstruct_row2(u);
  }
};

// 16-bit links: two rows kept (12 reals, row 2 rebuilt) unless TSM_LINK16_FULL
// is defined, in which case all 18 reals are stored:
//   12-real: [4][V] uint4 (U00 U01 U02 U10), then [4][V] uint2 (U11 U12)
//   18-real: [4][V] uint4 (U00 U01 U02 U10), [4][V] uint4 (U11 U12 U20 U21), [4][V] uint32 (U22)
template <bool BF>
struct Link16IO {
  __device__ __forceinline__ static float2 cvt(uint32_t w) { return BF ? b2f(w) : h2f(w); }
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int mu, int i, cplx<R> (&u)[3][3]) {
    const uint4* pa = reinterpret_cast<const uint4*>(base) + (size_t)mu * V + i;
    uint4 a = __ldg(pa);
    float2 t;
    t = cvt(a.x); u[0][0] = mk<R>(t.x, t.y);
    t = cvt(a.y); u[0][1] = mk<R>(t.x, t.y);
    t = cvt(a.z); u[0][2] = mk<R>(t.x, t.y);
    t = cvt(a.w); u[1][0] = mk<R>(t.x, t.y);
#ifdef TSM_LINK16_FULL
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(base) + 4 * V + (size_t)mu * V + i);
    const uint32_t c = __ldg(reinterpret_cast<const uint32_t*>(reinterpret_cast<const uint4*>(base) + 8 * V) +
                             (size_t)mu * V + i);
    t = cvt(b.x); u[1][1] = mk<R>(t.x, t.y);
    t = cvt(b.y); u[1][2] = mk<R>(t.x, t.y);
    t = cvt(b.z); u[2][0] = mk<R>(t.x, t.y);
    t = cvt(b.w); u[2][1] = mk<R>(t.x, t.y);
    t = cvt(c); u[2][2] = mk<R>(t.x, t.y);
#else
    const uint2* pb = reinterpret_cast<const uint2*>(reinterpret_cast<const uint4*>(base) + 4 * V) +
                      (size_t)mu * V + i;
    uint2 b = __ldg(pb);
    t = cvt(b.x); u[1][1] = mk<R>(t.x, t.y);
    t = cvt(b.y); u[1][2] = mk<R>(t.x, t.y);
    reconstruct_row2(u);
#endif
  }
};
template <>
struct LinkIO<TSM_F16> : Link16IO<false> {};
template <>
struct LinkIO<TSM_BF16> : Link16IO<true> {};

// float-float links: [4][9][V] float4 (re.hi, re.lo, im.hi, im.lo), all entries
template <>
struct LinkIO<TSM_DS> {
  template <typename R>
  __device__ __forceinline__ static void load(const void* base, size_t V, int mu, int i, cplx<R> (&u)[3][3]) {
    const float4* p = reinterpret_cast<const float4*>(base) + (size_t)mu * 9 * V + i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 d = __ldg(p + k * V);
      u[k / 3][k % 3] = mk<R>(from_pair<R>(d.x, d.y), from_pair<R>(d.z, d.w));
    }
  }
};

// bytes of one device gauge copy of precision p
inline size_t link_bytes(int p, size_t V) {
  switch (p) {
    case TSM_F64:
    case TSM_DS: return 4 * 9 * V * 16;
    case TSM_F32: return 4 * 3 * V * 16;
#ifdef TSM_LINK16_FULL
    default: return 4 * V * 16 * 2 + 4 * V * 4;
#else
    default: return 4 * V * 16 + 4 * V * 8;
#endif
  }
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block sum into double (fixed tree). `sh` needs blockDim/32 doubles.
template <typename T>
__device__ __forceinline__ double block_sum(T v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    s = (lane < nw) ? sh[lane] : 0.0;
    s = warp_sum(s);
  }
  return s;  // valid in thread 0
}

}  // namespace tsm
