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
#pragma once

#include "common.cuh"

namespace tsm {

constexpr int DSLASH_BS = 128;

struct DslashArgs {
  Geom g;
  const void* links;  // device links in the kernel's link precision
  const void* in;     // input field(s), native layout
  int nblk;           // blocks along the site axis
  int nrhs;           // right-hand sides in the launch
  double kappa;
  double tw;          // twist coefficient multiplying i g5
};

struct RedSlots {
  double* partial;    // [nrhs][nblk]
  unsigned* counter;  // [nrhs], zero between launches
};

// acc += (1 + S g_MU) W h(psi), W = U (DAG false) or U^dag (DAG true); sgn is
// the boundary sign of the link.
template <int MU, int S, bool DAG, typename R>
__device__ __forceinline__ void hop_dir(cplx<R> (&acc)[12], const cplx<R> (&p)[12], const cplx<R> (&u)[3][3],
                                        R sgn) {
  const R s = (R)S;
  cplx<R> h0[3], h1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cplx<R> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if (MU == 0) {          // h = psi_u - S i s1 psi_l
      h0[c] = p0 - s * times_i(p3);
      h1[c] = p1 - s * times_i(p2);
    } else if (MU == 1) {   // i s2 = [[0, 1], [-1, 0]]
      h0[c] = p0 - s * p3;
      h1[c] = p1 + s * p2;
    } else if (MU == 2) {   // i s3 = diag(i, -i)
      h0[c] = p0 - s * times_i(p2);
      h1[c] = p1 + s * times_i(p3);
    } else {                // g_t: h = psi_u + S psi_l
      h0[c] = p0 + s * p2;
      h1[c] = p1 + s * p3;
    }
  }
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
    w0[a] = sgn * w0[a];
    w1[a] = sgn * w1[a];
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

template <int MU, int SF, typename R, int PIN, int PL>
__device__ __forceinline__ void stencil_dir(cplx<R> (&acc)[12], const DslashArgs& a, int rhs, int i,
                                            const int c[4]) {
  const size_t V = (size_t)a.g.V;
  const int stride = dir_stride(a.g, MU);
  cplx<R> psi[12];
  cplx<R> u[3][3];
  // forward: (1 + SF g) U_mu(x) psi(x + mu)
  {
    const int n = fwd_site(a.g, i, c, MU, stride);
    SpinorIO<PIN>::load(a.in, V, rhs, n, psi);
    LinkIO<PL>::load(a.links, V, MU, i, u);
    const R sgn = (MU == 3 && c[3] == a.g.L[3] - 1) ? (R)a.g.bc : (R)1;
    hop_dir<MU, SF, false>(acc, psi, u, sgn);
  }
  // backward: (1 - SF g) U_mu(x - mu)^dag psi(x - mu)
  {
    const int n = bwd_site(a.g, i, c, MU, stride);
    SpinorIO<PIN>::load(a.in, V, rhs, n, psi);
    LinkIO<PL>::load(a.links, V, MU, n, u);
    const R sgn = (MU == 3 && c[3] == 0) ? (R)a.g.bc : (R)1;
    hop_dir<MU, -SF, true>(acc, psi, u, sgn);
  }
}

// Full operator at site i: out = in + i tw g5 in - kappa * hop.
template <int SF, typename R, int PIN, int PL>
__device__ __forceinline__ void apply_site(cplx<R> (&out)[12], const DslashArgs& a, int rhs, int i) {
  int c[4];
  site_coords(a.g, i, c);
  cplx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = mk<R>(0, 0);
  stencil_dir<0, SF, R, PIN, PL>(acc, a, rhs, i, c);
  stencil_dir<1, SF, R, PIN, PL>(acc, a, rhs, i, c);
  stencil_dir<2, SF, R, PIN, PL>(acc, a, rhs, i, c);
  stencil_dir<3, SF, R, PIN, PL>(acc, a, rhs, i, c);
  cplx<R> ctr[12];
  SpinorIO<PIN>::load(a.in, (size_t)a.g.V, rhs, i, ctr);
  const R kap = (R)a.kappa, tw = (R)a.tw;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const R g5 = (k < 6) ? (R)1 : (R)-1;
    cplx<R> t = ctr[k] + (g5 * tw) * times_i(ctr[k]);
    out[k] = t - kap * acc[k];
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
template <typename R, int SF, int PIN, int PL, class Epi>
__global__ void __launch_bounds__(DSLASH_BS) dslash_kernel(DslashArgs a, Epi epi) {
  __shared__ double sh[32];
  const int rhs = blockIdx.x % a.nrhs;
  const int blk = blockIdx.x / a.nrhs;
  if (!epi.active(rhs)) return;
  const int i = blk * DSLASH_BS + threadIdx.x;
  R red = (R)0;
  if (i < a.g.V) {
    cplx<R> out[12];
    apply_site<SF, R, PIN, PL>(out, a, rhs, i);
    red = epi.site(rhs, i, out);
  }
  if (Epi::kReduce) reduce_and_finalize(epi, epi.red, rhs, a.nblk, blk, (double)red, sh);
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

inline dim3 dslash_grid(int V, int nrhs) { return dim3((unsigned)((V + DSLASH_BS - 1) / DSLASH_BS) * nrhs, 1, 1); }

}  // namespace tsm
