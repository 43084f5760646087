// Field set-up kernels: gauge-copy packing, Z4 noise sources (Philox4x64-10)
// and conversions between the plain and the chunked spinor layouts.
#include <math.h>

#include <type_traits>

#include "internal.h"

namespace tsm {

namespace {

constexpr int BS = 256;

// ------------------------------------------------------------------ links
__global__ void pack_links_f64(const double2* __restrict__ src, double2* __restrict__ dst, int V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  for (int mu = 0; mu < 4; ++mu)
    for (int k = 0; k < 9; ++k) dst[((size_t)mu * 9 + k) * V + i] = src[((size_t)i * 4 + mu) * 9 + k];
}

// float-float copy of the FP64 links (precise operator of the reliable-update solver)
__global__ void pack_links_ds(const double2* __restrict__ src, float4* __restrict__ dst, int V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  for (int mu = 0; mu < 4; ++mu)
    for (int k = 0; k < 9; ++k) {
      const double2 u = src[((size_t)i * 4 + mu) * 9 + k];
      const dsf a(u.x), b(u.y);
      dst[((size_t)mu * 9 + k) * V + i] = make_float4(a.hi, a.lo, b.hi, b.lo);
    }
}

__global__ void pack_links_f32(const double2* __restrict__ src, float4* __restrict__ dst, int V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  for (int mu = 0; mu < 4; ++mu) {
    const double2* u = src + ((size_t)i * 4 + mu) * 9;  // row-major 3x3
    // rows 0 and 1: U00 U01 U02 U10 U11 U12
    dst[((size_t)mu * 3 + 0) * V + i] = make_float4((float)u[0].x, (float)u[0].y, (float)u[1].x, (float)u[1].y);
    dst[((size_t)mu * 3 + 1) * V + i] = make_float4((float)u[2].x, (float)u[2].y, (float)u[3].x, (float)u[3].y);
    dst[((size_t)mu * 3 + 2) * V + i] = make_float4((float)u[4].x, (float)u[4].y, (float)u[5].x, (float)u[5].y);
  }
}

template <bool BF>
__global__ void pack_links_16(const double2* __restrict__ src, uint4* __restrict__ dst, int V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  for (int mu = 0; mu < 4; ++mu) {
    const double2* u = src + ((size_t)i * 4 + mu) * 9;
    uint32_t w[9];
    for (int k = 0; k < 9; ++k)
      w[k] = BF ? f2b((float)u[k].x, (float)u[k].y) : f2h((float)u[k].x, (float)u[k].y);
    dst[(size_t)mu * V + i] = make_uint4(w[0], w[1], w[2], w[3]);
#ifdef TSM_LINK16_FULL
    dst[4 * (size_t)V + (size_t)mu * V + i] = make_uint4(w[4], w[5], w[6], w[7]);
    reinterpret_cast<uint32_t*>(dst + 8 * (size_t)V)[(size_t)mu * V + i] = w[8];
#else
    reinterpret_cast<uint2*>(dst + 4 * (size_t)V)[(size_t)mu * V + i] = make_uint2(w[4], w[5]);
#endif
  }
}

// ------------------------------------------------------------------ Philox4x64-10
// Salmon, Moraes, Dror, Shaw, SC'11: round (X0..X3) -> (hi(M1 X2) ^ X1 ^ K0,
// lo(M1 X2), hi(M0 X0) ^ X3 ^ K1, lo(M0 X0)); key += Weyl constants between rounds.
__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ void philox4x64_10(uint64_t (&x)[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t lo0 = M0 * x[0], hi0 = mulhi64(M0, x[0]);
    const uint64_t lo1 = M1 * x[2], hi1 = mulhi64(M1, x[2]);
    const uint64_t n0 = hi1 ^ x[1] ^ k0, n2 = hi0 ^ x[3] ^ k1;
    x[0] = n0;
    x[1] = lo1;
    x[2] = n2;
    x[3] = lo0;
  }
}

// Z4 sources; with t_first >= 0, field r is the source `first` kept on
// timeslice t_first + r (time dilution) and zero on every other timeslice.
template <int P>
__global__ void z4_kernel(uint64_t seed, uint64_t first, int V, void* out, int t_first = -1, int vol3 = 1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= V) return;
  const bool diluted = t_first >= 0;
  if (diluted && i / vol3 != t_first + r) {
    using R = ew_real<P>;
    cplx<R> z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) z[k] = mk<R>(0, 0);
    SpinorIO<P>::store(out, (size_t)V, r, i, z);
    return;
  }
  uint64_t x[4] = {(uint64_t)i, 0ull, 0ull, 0ull};
  philox4x64_10(x, seed, diluted ? first : first + (uint64_t)r);
  const uint64_t w = x[0];
  using R = ew_real<P>;
  cplx<R> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int z = (int)((w >> (2 * k)) & 3ull);
    // i^z: 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i
    v[k] = mk<R>((R)(z == 0 ? 1 : (z == 2 ? -1 : 0)), (R)(z == 1 ? 1 : (z == 3 ? -1 : 0)));
  }
  SpinorIO<P>::store(out, (size_t)V, r, i, v);
}

// The same Z4 sources split by parity for the even-odd solvers: site i of
// field r goes to odd or even at i >> 1 (all extents even), and the even
// sites also to diag_even as (cr + i ci g5) eta_e (M_ee^{-1} eta_e).  Every
// component of that product is exactly +-cr or +-ci, so float-float fields
// are computed in float-float (no FP64 work), the others in their own
// element-wise arithmetic.
template <int P>
__global__ void z4_eo_kernel(uint64_t seed, uint64_t first, Geom g, void* even, void* odd, void* diag_even, double cr,
                             double ci) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= g.V) return;
  uint64_t x[4] = {(uint64_t)i, 0ull, 0ull, 0ull};
  philox4x64_10(x, seed, first + (uint64_t)r);
  const uint64_t w = x[0];
  using R = typename std::conditional<P == TSM_DS, dsf, ew_real<P>>::type;
  cplx<R> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const int z = (int)((w >> (2 * k)) & 3ull);
    v[k] = mk<R>(R(z == 0 ? 1 : (z == 2 ? -1 : 0)), R(z == 1 ? 1 : (z == 3 ? -1 : 0)));
  }
  int c[4];
  site_coords(g, i, c);
  const size_t vh = (size_t)g.V / 2;
  if ((c[0] + c[1] + c[2] + c[3]) & 1) {
    SpinorIO<P>::store(odd, vh, r, i >> 1, v);
    return;
  }
  SpinorIO<P>::store(even, vh, r, i >> 1, v);
  const R a = R(cr), b = R(ci);
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = a * v[k] + (k < 6 ? b : -b) * times_i(v[k]);
  SpinorIO<P>::store(diag_even, vh, r, i >> 1, v);
}

// ------------------------------------------------------------------ layout conversions
template <int P>
__global__ void pack_kernel(const double2* __restrict__ plain, void* native, int V, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= V) return;
  cplx<double> v[12];
  const double2* p = plain + ((size_t)r * V + i) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = mk<double>(p[k].x * scale, p[k].y * scale);
  SpinorIO<P>::store(native, (size_t)V, r, i, v);
}

template <int P>
__global__ void unpack_kernel(const void* native, double2* __restrict__ plain, int V, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= V) return;
  cplx<double> v[12];
  SpinorIO<P>::load(native, (size_t)V, r, i, v);
  double2* p = plain + ((size_t)r * V + i) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = make_double2(v[k].re * scale, v[k].im * scale);
}

template <int PD, int PS>
__global__ void convert_kernel(void* dst, const void* src, int V, int gamma5) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= V) return;
  using R = ew_real<PD, PS>;
  cplx<R> v[12];
  SpinorIO<PS>::load(src, (size_t)V, r, i, v);
  if (gamma5) {
#pragma unroll
    for (int k = 6; k < 12; ++k) v[k] = mk<R>(-v[k].re, -v[k].im);
  }
  SpinorIO<PD>::store(dst, (size_t)V, r, i, v);
}

template <int PD>
int convert_from(int ps, void* dst, const void* src, int V, int nrhs, int gamma5, cudaStream_t s) {
  dim3 grid((V + BS - 1) / BS, nrhs);
  count_launches(1);
  switch (ps) {
    case TSM_F64: convert_kernel<PD, TSM_F64><<<grid, BS, 0, s>>>(dst, src, V, gamma5); break;
    case TSM_F32: convert_kernel<PD, TSM_F32><<<grid, BS, 0, s>>>(dst, src, V, gamma5); break;
    case TSM_F16: convert_kernel<PD, TSM_F16><<<grid, BS, 0, s>>>(dst, src, V, gamma5); break;
    case TSM_BF16: convert_kernel<PD, TSM_BF16><<<grid, BS, 0, s>>>(dst, src, V, gamma5); break;
    case TSM_DS: convert_kernel<PD, TSM_DS><<<grid, BS, 0, s>>>(dst, src, V, gamma5); break;
    default: return fail(TSM_ERR_INVALID_ARG, "bad precision %d", ps);
  }
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

}  // namespace

int build_links(tsm_gauge* g, const double* links_host) {
  const int V = g->geom.V;
  const size_t host_bytes = (size_t)V * 4 * 9 * sizeof(double2);
  DevBuf staging;
  TSM_TRY(staging.reserve(host_bytes));
  TSM_CUDA(cudaMemcpy(staging.p, links_host, host_bytes, cudaMemcpyHostToDevice));
  const int nb = (V + BS - 1) / BS;
  // an FP64 copy comes with its float-float twin
  if (has_prec(g, TSM_F64)) g->precisions |= 1u << TSM_DS;
  for (int p = 0; p <= TSM_DS; ++p) {
    if (!has_prec(g, p)) continue;
    TSM_TRY(g->links[p].reserve(link_bytes(p, V)));
    count_launches(1);
    const double2* src = staging.as<double2>();
    switch (p) {
      case TSM_F64: pack_links_f64<<<nb, BS>>>(src, g->links[p].as<double2>(), V); break;
      case TSM_F32: pack_links_f32<<<nb, BS>>>(src, g->links[p].as<float4>(), V); break;
      case TSM_F16: pack_links_16<false><<<nb, BS>>>(src, g->links[p].as<uint4>(), V); break;
      case TSM_BF16: pack_links_16<true><<<nb, BS>>>(src, g->links[p].as<uint4>(), V); break;
      case TSM_DS: pack_links_ds<<<nb, BS>>>(src, g->links[p].as<float4>(), V); break;
    }
    TSM_CUDA(cudaGetLastError());
  }
  TSM_CUDA(cudaDeviceSynchronize());
  return TSM_OK;
}

// ------------------------------------------------------------------ host gauge generator
// U = exp(i eps H), H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1): the eight
// normals of link (site i, direction mu) come from one Philox4x64-10 call
// (counter {4 i + mu, 0, 0, 0}, key {seed, 0x67617567}), its four words split
// into eight 32-bit uniforms u = (w + 1/2) / 2^32 and paired by Box-Muller.
// The exponential goes through the eigenvectors of H from cyclic Jacobi
// rotations (Golub and Van Loan, 8.5), in FP64.
namespace {

struct HC {
  double re, im;
};
inline HC hmul(HC a, HC b) { return HC{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline HC hconj(HC a) { return HC{a.re, -a.im}; }
inline HC hadd(HC a, HC b) { return HC{a.re + b.re, a.im + b.im}; }
inline HC hscale(HC a, double s) { return HC{a.re * s, a.im * s}; }

// Eigen-decomposition of a Hermitian 3x3 a = v diag(w) v^dag by cyclic Jacobi.
void jacobi_herm3(HC a[3][3], double w[3], HC v[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) v[i][j] = HC{i == j ? 1.0 : 0.0, 0.0};
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < 3; ++p)
      for (int q = p + 1; q < 3; ++q) off += a[p][q].re * a[p][q].re + a[p][q].im * a[p][q].im;
    if (off < 1e-34) break;
    for (int p = 0; p < 3; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const double mag = sqrt(a[p][q].re * a[p][q].re + a[p][q].im * a[p][q].im);
        if (mag < 1e-300) continue;
        // phase that makes a[p][q] real, then a real symmetric 2x2 rotation
        const HC ph = HC{a[p][q].re / mag, a[p][q].im / mag};
        const double theta = 0.5 * (a[q][q].re - a[p][p].re) / mag;
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        // J: columns p, q of the identity mixed: J[p][p] = c, J[q][q] = c,
        // J[p][q] = s ph, J[q][p] = -s conj(ph); a <- J^dag a J, v <- v J
        HC jpp{c, 0.0}, jqq{c, 0.0}, jpq = hscale(ph, s), jqp = hscale(hconj(ph), -s);
        for (int k = 0; k < 3; ++k) {  // a <- a J (columns p, q)
          const HC akp = a[k][p], akq = a[k][q];
          a[k][p] = hadd(hmul(akp, jpp), hmul(akq, jqp));
          a[k][q] = hadd(hmul(akp, jpq), hmul(akq, jqq));
          const HC vkp = v[k][p], vkq = v[k][q];
          v[k][p] = hadd(hmul(vkp, jpp), hmul(vkq, jqp));
          v[k][q] = hadd(hmul(vkp, jpq), hmul(vkq, jqq));
        }
        for (int k = 0; k < 3; ++k) {  // a <- J^dag a (rows p, q)
          const HC apk = a[p][k], aqk = a[q][k];
          a[p][k] = hadd(hmul(hconj(jpp), apk), hmul(hconj(jqp), aqk));
          a[q][k] = hadd(hmul(hconj(jpq), apk), hmul(hconj(jqq), aqk));
        }
      }
  }
  for (int i = 0; i < 3; ++i) w[i] = a[i][i].re;
}

}  // namespace

int generate_gauge_host(const int dims[4], double eps, uint64_t seed, double* out) {
  const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
  static const double kPi = 3.14159265358979323846;
  for (long long i = 0; i < V; ++i)
    for (int mu = 0; mu < 4; ++mu) {
      uint64_t x[4] = {(uint64_t)(4 * i + mu), 0ull, 0ull, 0ull};
      philox4x64_10(x, seed, 0x67617567ull);
      double u[8], h[8];
      for (int k = 0; k < 4; ++k) {
        u[2 * k] = ((double)(uint32_t)(x[k] & 0xffffffffu) + 0.5) * 0x1p-32;
        u[2 * k + 1] = ((double)(uint32_t)(x[k] >> 32) + 0.5) * 0x1p-32;
      }
      for (int k = 0; k < 4; ++k) {
        const double r = sqrt(-2.0 * log(u[2 * k])), ph = 2.0 * kPi * u[2 * k + 1];
        h[2 * k] = r * cos(ph);
        h[2 * k + 1] = r * sin(ph);
      }
      // H = sum_a h_a lambda_a / 2 (Gell-Mann basis)
      const double r3 = 1.0 / sqrt(3.0);
      HC a[3][3];
      a[0][0] = HC{0.5 * (h[2] + h[7] * r3), 0.0};
      a[1][1] = HC{0.5 * (-h[2] + h[7] * r3), 0.0};
      a[2][2] = HC{0.5 * (-2.0 * h[7] * r3), 0.0};
      a[0][1] = HC{0.5 * h[0], -0.5 * h[1]};
      a[0][2] = HC{0.5 * h[3], -0.5 * h[4]};
      a[1][2] = HC{0.5 * h[5], -0.5 * h[6]};
      a[1][0] = hconj(a[0][1]);
      a[2][0] = hconj(a[0][2]);
      a[2][1] = hconj(a[1][2]);
      double w[3];
      HC v[3][3];
      jacobi_herm3(a, w, v);
      double* o = out + ((size_t)i * 4 + mu) * 18;
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
          HC sum{0.0, 0.0};
          for (int k = 0; k < 3; ++k) {
            const HC e{cos(eps * w[k]), sin(eps * w[k])};
            sum = hadd(sum, hmul(hmul(v[r][k], e), hconj(v[c][k])));
          }
          o[2 * (3 * r + c)] = sum.re;
          o[2 * (3 * r + c) + 1] = sum.im;
        }
    }
  return TSM_OK;
}

int make_diluted_sources(const tsm_gauge* g, uint64_t seed, uint64_t source_id, int t_first, int n_t, int prec,
                         void* out, cudaStream_t s) {
  const int V = g->geom.V;
  const int vol3 = g->geom.L[0] * g->geom.L[1] * g->geom.L[2];
  dim3 grid((V + BS - 1) / BS, n_t);
  count_launches(1);
  switch (prec) {
    case TSM_F64: z4_kernel<TSM_F64><<<grid, BS, 0, s>>>(seed, source_id, V, out, t_first, vol3); break;
    case TSM_F32: z4_kernel<TSM_F32><<<grid, BS, 0, s>>>(seed, source_id, V, out, t_first, vol3); break;
    case TSM_F16: z4_kernel<TSM_F16><<<grid, BS, 0, s>>>(seed, source_id, V, out, t_first, vol3); break;
    case TSM_BF16: z4_kernel<TSM_BF16><<<grid, BS, 0, s>>>(seed, source_id, V, out, t_first, vol3); break;
    default: return fail(TSM_ERR_INVALID_ARG, "bad precision %d", prec);
  }
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

int make_sources(const tsm_gauge* g, uint64_t seed, uint64_t first, int nsrc, int prec, void* out,
                 cudaStream_t s) {
  const int V = g->geom.V;
  dim3 grid((V + BS - 1) / BS, nsrc);
  count_launches(1);
  switch (prec) {
    case TSM_F64: z4_kernel<TSM_F64><<<grid, BS, 0, s>>>(seed, first, V, out); break;
    case TSM_F32: z4_kernel<TSM_F32><<<grid, BS, 0, s>>>(seed, first, V, out); break;
    case TSM_F16: z4_kernel<TSM_F16><<<grid, BS, 0, s>>>(seed, first, V, out); break;
    case TSM_BF16: z4_kernel<TSM_BF16><<<grid, BS, 0, s>>>(seed, first, V, out); break;
    case TSM_DS: z4_kernel<TSM_DS><<<grid, BS, 0, s>>>(seed, first, V, out); break;
    default: return fail(TSM_ERR_INVALID_ARG, "bad precision %d", prec);
  }
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

int make_sources_eo(const tsm_gauge* g, uint64_t seed, uint64_t first, int nsrc, int prec, void* even, void* odd,
                    void* diag_even, double cr, double ci, cudaStream_t s) {
  const int V = g->geom.V;
  dim3 grid((V + BS - 1) / BS, nsrc);
  count_launches(1);
  switch (prec) {
    case TSM_F64: z4_eo_kernel<TSM_F64><<<grid, BS, 0, s>>>(seed, first, g->geom, even, odd, diag_even, cr, ci); break;
    case TSM_F32: z4_eo_kernel<TSM_F32><<<grid, BS, 0, s>>>(seed, first, g->geom, even, odd, diag_even, cr, ci); break;
    case TSM_DS: z4_eo_kernel<TSM_DS><<<grid, BS, 0, s>>>(seed, first, g->geom, even, odd, diag_even, cr, ci); break;
    default: return fail(TSM_ERR_INVALID_ARG, "bad precision %d for parity-split sources", prec);
  }
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

int spinor_pack(const tsm_gauge* g, int prec, const double* plain, void* native, int nrhs, double scale,
                cudaStream_t s) {
  const int V = g->geom.V;
  dim3 grid((V + BS - 1) / BS, nrhs);
  count_launches(1);
  const double2* src = reinterpret_cast<const double2*>(plain);
  switch (prec) {
    case TSM_F64: pack_kernel<TSM_F64><<<grid, BS, 0, s>>>(src, native, V, scale); break;
    case TSM_F32: pack_kernel<TSM_F32><<<grid, BS, 0, s>>>(src, native, V, scale); break;
    case TSM_F16: pack_kernel<TSM_F16><<<grid, BS, 0, s>>>(src, native, V, scale); break;
    case TSM_BF16: pack_kernel<TSM_BF16><<<grid, BS, 0, s>>>(src, native, V, scale); break;
    default: return fail(TSM_ERR_INVALID_ARG, "bad precision %d", prec);
  }
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

int spinor_unpack(const tsm_gauge* g, int prec, const void* native, double* plain, int nrhs, double scale,
                  cudaStream_t s) {
  const int V = g->geom.V;
  dim3 grid((V + BS - 1) / BS, nrhs);
  count_launches(1);
  double2* dst = reinterpret_cast<double2*>(plain);
  switch (prec) {
    case TSM_F64: unpack_kernel<TSM_F64><<<grid, BS, 0, s>>>(native, dst, V, scale); break;
    case TSM_F32: unpack_kernel<TSM_F32><<<grid, BS, 0, s>>>(native, dst, V, scale); break;
    case TSM_F16: unpack_kernel<TSM_F16><<<grid, BS, 0, s>>>(native, dst, V, scale); break;
    case TSM_BF16: unpack_kernel<TSM_BF16><<<grid, BS, 0, s>>>(native, dst, V, scale); break;
    default: return fail(TSM_ERR_INVALID_ARG, "bad precision %d", prec);
  }
  TSM_CUDA(cudaGetLastError());
  return TSM_OK;
}

int spinor_convert(const tsm_gauge* g, int pd, void* dst, int ps, const void* src, int nrhs, int gamma5,
                   cudaStream_t s) {
  const int V = g->geom.V;
  switch (pd) {
    case TSM_F64: return convert_from<TSM_F64>(ps, dst, src, V, nrhs, gamma5, s);
    case TSM_F32: return convert_from<TSM_F32>(ps, dst, src, V, nrhs, gamma5, s);
    case TSM_F16: return convert_from<TSM_F16>(ps, dst, src, V, nrhs, gamma5, s);
    case TSM_BF16: return convert_from<TSM_BF16>(ps, dst, src, V, nrhs, gamma5, s);
    case TSM_DS: return convert_from<TSM_DS>(ps, dst, src, V, nrhs, gamma5, s);
  }
  return fail(TSM_ERR_INVALID_ARG, "bad precision %d", pd);
}

}  // namespace tsm
