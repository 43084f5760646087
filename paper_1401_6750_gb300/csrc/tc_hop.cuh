// Checkerboarded hop of 16-bit fields on the tensor cores (warp-level
// mma.sync m16n8k16, 16-bit operands, FP32 accumulators) for batches of
// right-hand sides: the even-odd LP solver's sloppy operator (opt-in, see
// use_tc_hop below).
//
//   out(j) = (c0 + i c1 g5) center(j) + (h0 + i h1 g5) hop(in)(j)
//
// on the sites of parity a.parity (the coefficient form of dslash_eo_kernel,
// same epilogues).  hop = sum over the 8 hops of (1 + S g_mu) W psi(n), with
// W = U_mu(x) forward and U_mu(x - mu)^dag backward.
//
// The colour product W h of one hop, for the two projected spins h of every
// right-hand side, is a real matrix product: with R(W) = [[Re W, -Im W],
// [Im W, Re W]] (6 x 6) and h as 6 reals per spin,
//   [Re w; Im w] = R(W) [Re h; Im h].
// One mma.sync takes two sites: A holds R(W) of site 0 in rows/cols 0..5 and
// of site 1 in rows/cols 8..13 (zeros elsewhere), B the projected spinors of
// both sites' neighbours for 4 right-hand sides x 2 spins (columns
// n = 2 rhs + spin), C the upper spins.  The projector's lower spins are a
// spin-space map of w, which commutes with W, so a second mma.sync with the
// spin-mapped (and where needed i-rotated) h in B gives the lower spins
// directly.  28% of each tile is useful work; at the measured mma.sync rate
// that is still about twice the FP32 pipe, and the FP32 pipe would be left
// to the projections and the epilogue.
//
// CTA: 8 warps, TC_RHS = 8 right-hand sides, tiles of TC_TILE = 32 sites, and
// TC_TILES tiles per CTA (128 sites, the site blocking of the other stencils,
// so the reduction slots are the same).  Per hop the CTA stages in shared
// memory the projected half-spinors (and their i-rotation) of its 32 x 8
// (site, rhs) neighbours and R(W) of its 32 sites, then each warp runs the
// MMAs of two site pairs.  After 8 hops the accumulators go through shared
// memory so that one thread holds the 12 components of one (site, rhs) for
// the epilogue.
#pragma once

#include <stdlib.h>

#include "dslash.cuh"

namespace tsm {

constexpr int TC_TILE = 32;    // sites per tile
constexpr int TC_RHS = 8;      // right-hand sides per CTA
constexpr int TC_TILES = 4;    // tiles per CTA (TC_TILE * TC_TILES == DSLASH_BS)
constexpr int TC_BS = 256;     // threads per CTA
constexpr int TC_MIN_RHS = 8;  // smallest batch that takes this path
static_assert(TC_TILE * TC_TILES == DSLASH_BS, "tensor-core hop keeps the stencil site blocking");

// Shared memory of one CTA.  Staging (per hop) and the output exchange (per
// tile) are never live together.
struct TcStage {
  // projected half-spinor of (site, rhs): spin 0 in words 0..2, spin 1 in 3..5,
  // each spin as (Re h0, Re h1 | Re h2, Im h0 | Im h1, Im h2) = B rows 0..5
  uint32_t H[TC_TILE][TC_RHS][8];
  uint32_t HR[TC_TILE][TC_RHS][8];  // the same for i h
  uint32_t A[TC_TILE][8][4];        // R(W) rows 0..7 (6, 7 zero), 8 cols as 4 words
};
struct TcOut {
  float O[TC_TILE][TC_RHS][25];  // hop sum of (site, rhs): 12 complex, + 1 pad
};
union TcSmem {
  TcStage st;
  TcOut out;
};

__device__ __forceinline__ uint32_t neg2(uint32_t x) { return x ^ 0x80008000u; }

template <bool BF>
__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  return BF ? f2b(lo, hi) : f2h(lo, hi);
}

template <bool BF>
__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a3, uint32_t b0, uint32_t b1) {
  const uint32_t z = 0u;
  if (BF) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(z), "r"(z), "r"(a3), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(z), "r"(z), "r"(a3), "r"(b0), "r"(b1));
  }
}

// Stage one hop: projected spinors for (site s = tid & 31, rhs r = tid >> 5)
// and R(W) row g = tid & 7 of site tid >> 3.
template <int MU, bool FWD, int SF, bool BF>
__device__ __forceinline__ void tc_stage(TcStage& sm, const DslashArgs& a, int r0, unsigned act_mask, int tile0,
                                         const int (&ch)[4], int ih, bool vh, const int (&ca)[4], int ia, bool va) {
  constexpr int S = FWD ? SF : -SF;  // projector sign of this hop
  const size_t V = (size_t)a.g.V;
  const size_t FS = V / 2;
  const int stride = dir_stride(a.g, MU);
  const int tid = threadIdx.x;
  {  // spinors
    const int s = tid & 31, r = tid >> 5;
    uint32_t w[6] = {0, 0, 0, 0, 0, 0}, x[6] = {0, 0, 0, 0, 0, 0};
    if (vh && ((act_mask >> r) & 1u)) {
      const int n = FWD ? fwd_site(a.g, ih, ch, MU, stride) : bwd_site(a.g, ih, ch, MU, stride);
      const uint4* p = reinterpret_cast<const uint4*>(a.in) + (size_t)(r0 + r) * 3 * FS + (n >> 1);
      const uint4 u0 = __ldg(p), u1 = __ldg(p + FS), u2 = __ldg(p + 2 * FS);
      const uint32_t v[12] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
      using P2 = Packed2<BF>;
      auto add = [](uint32_t x, uint32_t y) { return P2::add(x, y); };
      auto sub = [](uint32_t x, uint32_t y) { return P2::sub(x, y); };
      auto muli = [](uint32_t x) { return P2::muli(x); };
      uint32_t q0[3], q1[3];
#pragma unroll
      for (int col = 0; col < 3; ++col)
        project_pair<MU, S>(q0[col], q1[col], v[col], v[3 + col], v[6 + col], v[9 + col], add, sub, muli);
      // B rows of one spin: (Re h0, Re h1), (Re h2, Im h0), (Im h1, Im h2); half2 words hold (re, im)
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        const uint32_t h[3] = {sp ? q1[0] : q0[0], sp ? q1[1] : q0[1], sp ? q1[2] : q0[2]};
        w[3 * sp + 0] = __byte_perm(h[0], h[1], 0x5410);
        w[3 * sp + 1] = __byte_perm(h[2], h[0], 0x7610);
        w[3 * sp + 2] = __byte_perm(h[1], h[2], 0x7632);
        // i h = (-Im h, Re h)
        x[3 * sp + 0] = neg2(__byte_perm(h[0], h[1], 0x7632));
        x[3 * sp + 1] = __byte_perm(h[2], h[0], 0x5432) ^ 0x00008000u;
        x[3 * sp + 2] = __byte_perm(h[1], h[2], 0x5410);
      }
    }
    uint4* dh = reinterpret_cast<uint4*>(&sm.H[s][r][0]);
    uint4* dx = reinterpret_cast<uint4*>(&sm.HR[s][r][0]);
    dh[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dh[1] = make_uint4(w[4], w[5], 0u, 0u);
    dx[0] = make_uint4(x[0], x[1], x[2], x[3]);
    dx[1] = make_uint4(x[4], x[5], 0u, 0u);
  }
  {  // R(W) row g of site sa
    const int sa = tid >> 3, g = tid & 7;
    uint32_t row[4] = {0u, 0u, 0u, 0u};
    if (va && g < 6) {
      const int ls = FWD ? ia : bwd_site(a.g, ia, ca, MU, stride);  // link site
      cplx<float> u[3][3];
      LinkIO<BF ? TSM_BF16 : TSM_F16>::load(a.links, V, MU, ls, u);
      const bool edge = (MU == 3) && (FWD ? (ca[3] == a.g.L[3] - 1) : (ca[3] == 0));
      const float sg = (edge && a.g.bc < 0) ? -1.0f : 1.0f;
      const int rr = g / 3, ar = g % 3;  // row: real (0) or imaginary (1) part of colour ar
      float e[8];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // W[ar][b] = U[ar][b] (forward) or conj(U[b][ar]) (backward); the
        // selects keep the register indices static
        cplx<float> x[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) x[c] = FWD ? u[c][b] : conjc(u[b][c]);
        const cplx<float> wv = (ar == 0) ? x[0] : (ar == 1 ? x[1] : x[2]);
        e[b] = sg * (rr == 0 ? wv.re : wv.im);       // cols 0..2: Re h
        e[3 + b] = sg * (rr == 0 ? -wv.im : wv.re);  // cols 3..5: Im h
      }
      e[6] = e[7] = 0.0f;
      row[0] = pack_half2<BF>(e[0], e[1]);
      row[1] = pack_half2<BF>(e[2], e[3]);
      row[2] = pack_half2<BF>(e[4], e[5]);
      row[3] = 0u;
    }
    *reinterpret_cast<uint4*>(&sm.A[sa][g][0]) = make_uint4(row[0], row[1], row[2], row[3]);
  }
}

// The MMAs of one hop for warp w: site pairs p = w and w + 8 (sites 2p, 2p+1),
// column tiles c = 0, 1 (right-hand sides 4c .. 4c+3).
template <int MU, bool FWD, int SF, bool BF>
__device__ __forceinline__ void tc_mma(const TcStage& sm, float (&cu)[2][2][4], float (&cl)[2][2][4]) {
  constexpr int S = FWD ? SF : -SF;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // lower spins: column (rhs, s') of B' = f h_{src spin}, f in {+-1, +-i}
  //   x: s'=0: S i h1, s'=1: S i h0     y: s'=0: S h1,  s'=1: -S h0
  //   z: s'=0: S i h0, s'=1: -S i h1    t: s'=0: S h0,  s'=1: S h1
  const int sp = g & 1;
  const bool rot = (MU == 0 || MU == 2);
  const int src = (MU == 0 || MU == 1) ? 1 - sp : sp;
  const bool neg = (S < 0) != ((MU == 1 || MU == 2) && sp == 1);
#pragma unroll
  for (int pp = 0; pp < 2; ++pp) {
    const int p = w + 8 * pp;
    const uint32_t a0 = sm.A[2 * p][g][t], a3 = sm.A[2 * p + 1][g][t];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int rl = 4 * c + (g >> 1);
      uint32_t b0 = 0u, b1 = 0u, l0 = 0u, l1 = 0u;
      if (t < 3) {
        b0 = sm.H[2 * p][rl][3 * sp + t];
        b1 = sm.H[2 * p + 1][rl][3 * sp + t];
        l0 = rot ? sm.HR[2 * p][rl][3 * src + t] : sm.H[2 * p][rl][3 * src + t];
        l1 = rot ? sm.HR[2 * p + 1][rl][3 * src + t] : sm.H[2 * p + 1][rl][3 * src + t];
        if (neg) {
          l0 = neg2(l0);
          l1 = neg2(l1);
        }
      }
      mma16816<BF>(cu[pp][c], a0, a3, b0, b1);
      mma16816<BF>(cl[pp][c], a0, a3, l0, l1);
    }
  }
}

template <int MU, bool FWD, int SF, bool BF>
__device__ __forceinline__ void tc_hop(TcSmem& sm, const DslashArgs& a, int r0, unsigned act_mask, int tile0,
                                       const int (&ch)[4], int ih, bool vh, const int (&ca)[4], int ia, bool va,
                                       float (&cu)[2][2][4], float (&cl)[2][2][4]) {
  tc_stage<MU, FWD, SF, BF>(sm.st, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va);
  __syncthreads();
  tc_mma<MU, FWD, SF, BF>(sm.st, cu, cl);
  __syncthreads();
}

// a.nblk must be ceil(V/2 / DSLASH_BS); the grid is a.nblk x ceil(nrhs / TC_RHS)
// with the right-hand-side group fastest.
template <int SF, int PIN, class Epi>
__global__ void __launch_bounds__(TC_BS, 2) tc_hop_eo_kernel(DslashArgs a, Epi epi) {
  constexpr bool BF = (PIN == TSM_BF16);
  __shared__ __align__(16) TcSmem sm;
  __shared__ bool is_last;
  const int ngrp = (a.nrhs + TC_RHS - 1) / TC_RHS;
  const int grp = blockIdx.x % ngrp;
  const int blk = blockIdx.x / ngrp;
  const int r0 = grp * TC_RHS;
  unsigned act_mask = 0u;
#pragma unroll
  for (int r = 0; r < TC_RHS; ++r)
    if (r0 + r < a.nrhs && epi.active(r0 + r)) act_mask |= 1u << r;
  if (act_mask == 0u) return;  // uniform over the group's CTAs
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int Vh = a.g.V / 2;
  const size_t FS = (size_t)Vh;
  const int my_rhs = r0 + w;  // the epilogue's right-hand side (warp w)
  const bool my_act = (act_mask >> w) & 1u;
  float red = 0.0f;
#pragma unroll 1
  for (int tile = 0; tile < TC_TILES; ++tile) {
    const int tile0 = blk * DSLASH_BS + tile * TC_TILE;
    // sites of the two staging roles: spinors (tid & 31), links (tid >> 3)
    int ch[4], ca[4];
    const int jh = tile0 + (tid & 31), ja = tile0 + (tid >> 3);
    const bool vh = jh < Vh, va = ja < Vh;
    const int ih = vh ? eo_site(a.g, jh, a.parity, ch) : 0;
    const int ia = va ? eo_site(a.g, ja, a.parity, ca) : 0;
    if (!vh) ch[0] = ch[1] = ch[2] = ch[3] = 0;
    if (!va) ca[0] = ca[1] = ca[2] = ca[3] = 0;
    float cu[2][2][4], cl[2][2][4];
#pragma unroll
    for (int pp = 0; pp < 2; ++pp)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) cu[pp][c][k] = cl[pp][c][k] = 0.0f;
    tc_hop<0, true, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    tc_hop<0, false, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    tc_hop<1, true, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    tc_hop<1, false, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    tc_hop<2, true, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    tc_hop<2, false, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    tc_hop<3, true, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    tc_hop<3, false, SF, BF>(sm, a, r0, act_mask, tile0, ch, ih, vh, ca, ia, va, cu, cl);
    // accumulators -> (site, rhs) rows: thread (g, t) of warp w holds, for
    // pair p and column tile c, row g (= re/im g / 3, colour g % 3) of sites
    // 2p (c[0], c[1]) and 2p + 1 (c[2], c[3]), spins 0 and 1 of rhs 4c + t
    {
      const int g = lane >> 2, t = lane & 3;
      if (g < 6) {
        const int ri = g / 3, col = g % 3;
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          const int p = w + 8 * pp;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int rl = 4 * c + t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {  // site 2p + h
              float* o = sm.out.O[2 * p + h][rl];
              o[2 * col + ri] = cu[pp][c][2 * h];             // spin 0
              o[2 * (3 + col) + ri] = cu[pp][c][2 * h + 1];   // spin 1
              o[2 * (6 + col) + ri] = cl[pp][c][2 * h];       // spin 2
              o[2 * (9 + col) + ri] = cl[pp][c][2 * h + 1];   // spin 3
            }
          }
        }
      }
    }
    __syncthreads();
    {  // epilogue of (site lane, rhs w)
      const int j = tile0 + lane;
      if (j < Vh && my_act) {
        const float* o = sm.out.O[lane][w];
        cplx<float> out[12], ctr[12];
        float c0, c1, h0, h1;
        EoCoef<float>::get(a, c0, c1, h0, h1);
        if (a.center) {
          SpinorIO<PIN>::load(a.center, FS, my_rhs, j, ctr);
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) ctr[k] = mk<float>(0, 0);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float g5 = (k < 6) ? 1.0f : -1.0f;
          const cplx<float> hv = mk<float>(o[2 * k], o[2 * k + 1]);
          out[k] = c0 * ctr[k] + (g5 * c1) * times_i(ctr[k]) + h0 * hv + (g5 * h1) * times_i(hv);
        }
        red += epi.site(my_rhs, j, out);
      }
    }
    __syncthreads();
  }
  if (Epi::kReduce) {
    // per-rhs partial of this CTA (warp w = rhs r0 + w), then the last CTA of
    // the group sums every CTA's partial in a fixed order
    const double v = warp_sum((double)red);
    if (lane == 0 && my_act) {
      epi.red.partial[(size_t)my_rhs * a.nblk + blk] = v;
      __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
      const unsigned t = atomicAdd(&epi.red.counter[r0], 1u);
      is_last = (t == (unsigned)(a.nblk - 1));
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      if (my_act) {
        const double* pr = epi.red.partial + (size_t)my_rhs * a.nblk;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int q = lane;
        for (; q + 96 < a.nblk; q += 128) {
          s0 += __ldcg(pr + q);
          s1 += __ldcg(pr + q + 32);
          s2 += __ldcg(pr + q + 64);
          s3 += __ldcg(pr + q + 96);
        }
        for (; q < a.nblk; q += 32) s0 += __ldcg(pr + q);
        double s = warp_sum((s0 + s1) + (s2 + s3));
        if (lane == 0) epi.finalize(my_rhs, s);
      }
      if (tid == 0) epi.red.counter[r0] = 0u;
    }
  }
}

// Opt-in (TSM_TC_HOP=1 in the environment): measured on one GB300 at
// 24^3x48 with 32 right-hand sides, this kernel is 4.3x slower than the
// CUDA-core stencil (step A 486 against 2079 GB/s).  Each of its 32 hop
// phases per CTA waits on its own global loads between barriers with 16 warps
// resident, and the link fragments, built per 8 right-hand sides, cost most
// of the instructions the MMAs save.  It stays as a verified starting point
// for a pipelined form (asynchronous copies of the next hop's data, 32
// right-hand sides per CTA).
inline bool use_tc_hop() {
  static const bool on = [] {
    const char* e = getenv("TSM_TC_HOP");
    return e && e[0] == '1';
  }();
  return on;
}

// launch_dslash_eo, with 16-bit batches of at least TC_MIN_RHS right-hand
// sides on the tensor cores when TSM_TC_HOP=1.  a.nblk must be
// ceil(V/2 / DSLASH_BS).
template <typename R, int SF, int PIN, int PL, class Epi>
inline void launch_dslash_eo_tc(int nr, const DslashArgs& a, const Epi& e, cudaStream_t s) {
  if constexpr ((PIN == TSM_F16 || PIN == TSM_BF16) && PL == PIN && std::is_same<R, float>::value) {
    if (a.nrhs >= TC_MIN_RHS && use_tc_hop()) {
      const unsigned grid = (unsigned)a.nblk * (unsigned)((a.nrhs + TC_RHS - 1) / TC_RHS);
      tc_hop_eo_kernel<SF, PIN, Epi><<<grid, TC_BS, 0, s>>>(a, e);
      return;
    }
  }
  launch_dslash_eo<R, SF, PIN, PL>(nr, a, e, s);
}

}  // namespace tsm
