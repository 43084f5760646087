// Solver building blocks shared by the single-instance CG (solver.cu) and the
// multi-instance CG (batch.cu): precision traits, the per-site epilogues of
// the fused CG kernels and the element-wise kernels.  See solver.cu for the
// algorithm.
#pragma once

#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <type_traits>

#include "dslash.cuh"
#include "internal.h"

namespace tsm {
namespace solverk {

constexpr int EW_BS = 256;

struct SolveParams {
  double rho2;
  double delta2;
  double inv_ncomp;  // 1 / (12 V)
  int max_iter;
  int scaled;
};

template <int KIND>
struct Traits;
// Rs / Rp: arithmetic of the sloppy / precise operator; PS, PA, PP: storage of
// p and Ap, of x and r, and of b and the precise operator's fields; PLs, PLp:
// link copies; PX: input of the precise operator (x, or the accumulated
// solution when XACC); PXA: storage of that accumulator.
template <>
struct Traits<TSM_SOLVER_F64> {
  using Rs = double;
  using Rp = double;
  static constexpr int PS = TSM_F64, PA = TSM_F64, PP = TSM_F64, PLs = TSM_F64, PLp = TSM_F64, PX = TSM_F64;
  static constexpr int PXA = TSM_F64;
  static constexpr bool XACC = false, SCALED = false;
  static constexpr double DELTA = 0.0;
  static constexpr double CERT = 1e-6;  // certification margin (see cert_rho)
};
// The precise side works in float-float (about 44-bit significands): the true
// residual it certifies is many decades below rho = 1e-8, and GB300 runs it
// on the FP32 pipes instead of its narrow FP64 unit.
template <>
struct Traits<TSM_SOLVER_F32_RELIABLE> {
  using Rs = float;
  using Rp = dsf;
  static constexpr int PS = TSM_F32, PA = TSM_F32, PP = TSM_DS, PLs = TSM_F32, PLp = TSM_DS, PX = TSM_DS;
  static constexpr int PXA = TSM_DS;
  static constexpr bool XACC = true, SCALED = false;
  // FP32 recurrences stay accurate over four decades below the last true
  // residual (24^3 x 48, rho 1e-8: the same iterations as 1e-3, one
  // replacement fewer)
  static constexpr double DELTA = 1e-4;
  static constexpr double CERT = 1e-2;
};
template <>
struct Traits<TSM_SOLVER_LP_F16> {
  using Rs = float;
  using Rp = float;
  static constexpr int PS = TSM_F16, PA = TSM_F32, PP = TSM_F32, PLs = TSM_F16, PLp = TSM_F32, PX = TSM_F32;
  static constexpr int PXA = TSM_F32;
  static constexpr bool XACC = false, SCALED = true;
  static constexpr double DELTA = 0.1;
  static constexpr double CERT = 1e-3;
};
template <>
struct Traits<TSM_SOLVER_LP_BF16> {
  using Rs = float;
  using Rp = float;
  static constexpr int PS = TSM_BF16, PA = TSM_F32, PP = TSM_F32, PLs = TSM_BF16, PLp = TSM_F32, PX = TSM_F32;
  static constexpr int PXA = TSM_F32;
  static constexpr bool XACC = false, SCALED = true;
  static constexpr double DELTA = 0.1;
  static constexpr double CERT = 1e-3;
};

// The target the solvers stop at: rho (1 - CERT).  The true residual the
// solver reports is computed by its precise operator (FP64, float-float or
// FP32 links and arithmetic) and differs from the exact FP64 value of the
// returned solution by that operator's rounding; CERT is a margin for it, so
// that the exact true residual of every returned solution is at most rho.
// Measured differences, reported against the oracle's FP64 recomputation, on
// 4^4 to 24^3 x 48 lattices: below 3e-7 relative for the FP32 precise
// operator (LP maps) and the float-float one (HP map); CERT leaves a factor
// of more than 1000 (FP32: 1e-3) and 30000 (float-float: 1e-2) on top.  The
// float-float margin is wider because its rounding, relative to the residual,
// grows as rho falls (a few 1e-12 |b| in absolute terms).
__host__ __device__ inline double cert_rho(double rho, double margin) { return rho * (1.0 - margin); }

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// ---------------------------------------------------------------- epilogues
// b = M^dag eta; |b|^2 initialises the state of each right-hand side.
template <typename R, int PO>
struct EpiInitB {
  static constexpr bool kReduce = true;
  void* out;
  size_t V;
  RhsState* st;
  RedSlots red;
  SolveParams prm;
  __device__ bool active(int) const { return true; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    SpinorIO<PO>::store(out, V, rhs, i, o);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) n += norm2(o[k]);
    return n;
  }
  __device__ void finalize(int rhs, double bb) const {
    RhsState& s = st[rhs];
    s.bb = bb;
    s.rho2bb = prm.rho2 * bb;
    s.rr = bb;
    s.r_max2 = bb;
    s.true_rr = bb;
    s.delta2 = prm.delta2;
    s.alpha = s.beta = 0.0;
    s.sigma = (prm.scaled && bb > 0.0) ? sqrt(bb * prm.inv_ncomp) : 1.0;
    s.c_r = 1.0 / s.sigma;
    s.c_p = 0.0;
    s.iter = 0;
    s.max_iter = prm.max_iter;
    s.need_ru = 0;
    s.n_ru = 0;
    s.restarts = 0;
    s.restart_p = 0;
    if (!finite_d(bb)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
    } else if (bb == 0.0) {
      s.status = ST_DONE;
      s.active = 0;
    } else {
      s.status = ST_RUNNING;
      s.active = 1;
    }
  }
};

// q = M p (sloppy), |q|^2 -> alpha.
template <typename R, int PQ>
struct EpiMp {
  static constexpr bool kReduce = true;
  void* q;
  size_t V;
  RhsState* st;
  RedSlots red;
  __device__ bool active(int rhs) const { return st[rhs].active != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    SpinorIO<PQ>::store(q, V, rhs, i, o);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) n += norm2(o[k]);
    return n;
  }
  __device__ void finalize(int rhs, double qq) const {
    RhsState& s = st[rhs];
    s.restart_p = 0;
    const double pap = s.sigma * s.sigma * qq;
    if (!(pap > 0.0) || !finite_d(pap)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
      return;
    }
    s.alpha = s.rr / pap;
  }
};

// Ap = M^dag q (sloppy); r -= alpha Ap; x += alpha p; |r|^2 -> beta, stop test.
template <typename R, int PA, int PS>
struct EpiCG {
  static constexpr bool kReduce = true;
  void* r;
  void* x;
  const void* p;
  size_t V;
  RhsState* st;
  RedSlots red;
  SolveParams prm;
  __device__ bool active(int rhs) const { return st[rhs].active != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&ap)[12]) const {
    const R a = (R)(st[rhs].alpha * st[rhs].sigma);
    cplx<R> rv[12], xv[12], pv[12];
    SpinorIO<PA>::load(r, V, rhs, i, rv);
    SpinorIO<PA>::load(x, V, rhs, i, xv);
    SpinorIO<PS>::load(p, V, rhs, i, pv);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rv[k] = rv[k] - a * ap[k];
      xv[k] = xv[k] + a * pv[k];
      n += norm2(rv[k]);
    }
    SpinorIO<PA>::store(r, V, rhs, i, rv);
    SpinorIO<PA>::store(x, V, rhs, i, xv);
    return n;
  }
  __device__ void finalize(int rhs, double rr_new) const {
    RhsState& s = st[rhs];
    s.iter += 1;
    if (!finite_d(rr_new)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
      return;
    }
    const double beta = rr_new / s.rr;
    s.beta = beta;
    s.rr = rr_new;
    if (rr_new > s.r_max2) s.r_max2 = rr_new;
    double sig = 1.0;
    if (prm.scaled) {
      sig = sqrt(rr_new * prm.inv_ncomp);
      if (!(sig > 0.0)) sig = 1.0;
    }
    s.c_r = 1.0 / sig;
    s.c_p = beta * s.sigma / sig;
    s.sigma = sig;
    if (rr_new <= s.rho2bb) {
      s.status = ST_ITER_CONV;
      s.active = 0;
    } else if (s.iter >= s.max_iter) {
      s.status = ST_MAXITER;
      s.active = 0;
    } else if (s.delta2 > 0.0 && rr_new < s.delta2 * s.r_max2) {
      s.need_ru = 1;
    }
  }
};

// t = M x with the precise operator, for the rhs in mask.
template <typename R, int PO>
struct EpiStoreMasked {
  static constexpr bool kReduce = false;
  void* out;
  size_t V;
  const int* mask;
  RedSlots red;
  __device__ bool active(int rhs) const { return mask[rhs] != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    SpinorIO<PO>::store(out, V, rhs, i, o);
    return (R)0;
  }
  __device__ void finalize(int, double) const {}
};

// r = b - M^dag t (precise); |r|^2 is the true residual.
template <typename R, int PB, int PA>
struct EpiResidual {
  static constexpr bool kReduce = true;
  const void* b;
  void* r;
  size_t V;
  const int* mask;
  RhsState* st;
  RedSlots red;
  SolveParams prm;
  __device__ bool active(int rhs) const { return mask[rhs] != 0; }
  __device__ R site(int rhs, int i, cplx<R> (&o)[12]) const {
    cplx<R> bv[12];
    SpinorIO<PB>::load(b, V, rhs, i, bv);
    R n = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      bv[k] = bv[k] - o[k];
      n += norm2(bv[k]);
    }
    SpinorIO<PA>::store(r, V, rhs, i, bv);
    return n;
  }
  __device__ void finalize(int rhs, double rr) const {
    RhsState& s = st[rhs];
    s.true_rr = rr;
    s.rr = rr;
    s.r_max2 = rr;
    s.need_ru = 0;
    s.n_ru += 1;
    if (!finite_d(rr)) {
      s.status = ST_BREAKDOWN;
      s.active = 0;
      return;
    }
    if (s.status == ST_ITER_CONV || s.status == ST_MAXITER) {
      if (rr <= s.rho2bb) {
        s.status = ST_DONE;
        s.active = 0;
      } else if (s.status == ST_MAXITER || s.iter >= s.max_iter) {
        s.status = ST_FAILED;
        s.active = 0;
      } else {
        // restart from the true residual: p = r
        s.status = ST_RUNNING;
        s.active = 1;
        s.restarts += 1;
        s.restart_p = 1;
        double sig = 1.0;
        if (prm.scaled) {
          sig = sqrt(rr * prm.inv_ncomp);
          if (!(sig > 0.0)) sig = 1.0;
        }
        s.c_r = 1.0 / sig;
        s.c_p = 0.0;
        s.sigma = sig;
      }
    }
  }
};

// ---------------------------------------------------------------- elementwise kernels
template <int PB, int PA, int PS, bool XACC, int PXA>
__global__ void k_init(const void* b, void* r, void* x, void* p, void* xacc, const RhsState* st, int V) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (i >= V) return;
  using R = ew_real<PB, PA, PS, (XACC ? PXA : PA)>;
  cplx<R> v[12], z[12];
  SpinorIO<PB>::load(b, (size_t)V, rhs, i, v);
#pragma unroll
  for (int k = 0; k < 12; ++k) z[k] = mk<R>(0, 0);
  SpinorIO<PA>::store(r, (size_t)V, rhs, i, v);
  SpinorIO<PA>::store(x, (size_t)V, rhs, i, z);
  if (XACC) SpinorIO<PXA>::store(xacc, (size_t)V, rhs, i, z);
  const R c = (R)st[rhs].c_r;
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = c * v[k];
  SpinorIO<PS>::store(p, (size_t)V, rhs, i, v);
}

// p = c_r r + c_p p for rhs with (mode 0) active or (mode 1) restart_p set;
// coefficients in FP64 for the all-FP64 solver, FP32 otherwise.
template <int PA, int PS>
__global__ void k_pupdate(const void* r, void* p, const RhsState* st, int mode, int V) {
  using Rq = typename std::conditional<PA == TSM_F64 && PS == TSM_F64, double, float>::type;
  const int rhs = blockIdx.y;
  const RhsState& s = st[rhs];
  if (mode == 0 ? !s.active : !s.restart_p) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const Rq cr = (Rq)s.c_r, cp = (Rq)s.c_p;
  cplx<Rq> rv[12], pv[12];
  SpinorIO<PA>::load(r, (size_t)V, rhs, i, rv);
  SpinorIO<PS>::load(p, (size_t)V, rhs, i, pv);
#pragma unroll
  for (int k = 0; k < 12; ++k) pv[k] = cr * rv[k] + cp * pv[k];
  SpinorIO<PS>::store(p, (size_t)V, rhs, i, pv);
}

// xacc += x; x = 0 (masked): fold the sloppy solution into the accumulator.
template <int PA, int PXA>
__global__ void k_fold(void* x, void* xacc, const int* mask, int V) {
  const int rhs = blockIdx.y;
  if (!mask[rhs]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  using R = ew_real<PA, PXA>;
  cplx<R> xv[12], av[12];
  SpinorIO<PA>::load(x, (size_t)V, rhs, i, xv);
  SpinorIO<PXA>::load(xacc, (size_t)V, rhs, i, av);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    av[k] = av[k] + xv[k];
    xv[k] = mk<R>(0, 0);
  }
  SpinorIO<PXA>::store(xacc, (size_t)V, rhs, i, av);
  SpinorIO<PA>::store(x, (size_t)V, rhs, i, xv);
}

template <int PA, int PO, bool XACC, int PXA>
__global__ void k_output(const void* x, const void* xacc, void* out, int gamma5, int V) {
  const int rhs = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V) return;
  using R = ew_real<PA, PO, (XACC ? PXA : PA)>;
  cplx<R> v[12];
  SpinorIO<PA>::load(x, (size_t)V, rhs, i, v);
  if (XACC) {
    cplx<R> a[12];
    SpinorIO<PXA>::load(xacc, (size_t)V, rhs, i, a);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = v[k] + a[k];
  }
  if (gamma5) {
#pragma unroll
    for (int k = 6; k < 12; ++k) v[k] = mk<R>(-v[k].re, -v[k].im);
  }
  SpinorIO<PO>::store(out, (size_t)V, rhs, i, v);
}

inline size_t field_bytes(int prec, int V, int nrhs) { return (size_t)nrhs * spinor_chunks(prec) * (size_t)V * 16; }

}  // namespace solverk
}  // namespace tsm
