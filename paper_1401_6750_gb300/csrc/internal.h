// Host-side internals shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tsm.h"

namespace tsm {

// Record a message for tsm_last_error() and return `code`.
int fail(int code, const char* fmt, ...);
int cuda_status(cudaError_t e, const char* what, const char* file, int line);

#define TSM_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::tsm::cuda_status(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define TSM_TRY(expr)            \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != TSM_OK) return rc_; \
  } while (0)

// Owning device allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  // Grow to at least n bytes (contents are not kept).
  int reserve(size_t n);
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Orders the uses of a library-owned buffer across streams: a user's stream
// waits (enter) for the event recorded after the previous user's last
// launch, and records it again (leave) after its own.  Callers hold the
// buffer's mutex from enter to leave.  Inside a stream capture both steps
// are left out (an event recorded outside a capture cannot be waited on
// inside it); captured calls on one handle must then be ordered by the
// caller.
struct UseOrder {
  cudaEvent_t done = nullptr;
  bool capturing = false;
  UseOrder() = default;
  UseOrder(const UseOrder&) = delete;
  UseOrder& operator=(const UseOrder&) = delete;
  ~UseOrder() {
    if (done) cudaEventDestroy(done);
  }
  int enter(cudaStream_t st);
  int leave(cudaStream_t st);
  // host wait for the previous user's last launch (before freeing or growing)
  int wait_host();
};

// Library-owned scratch that calls on any host thread and stream share.  A
// call holds the lease (and so the mutex) while it enqueues the work that
// uses the buffer, ordered as UseOrder describes.
struct SharedScratch {
  std::mutex mu;
  DevBuf buf;
  UseOrder order;
};

class ScratchLease {
 public:
  explicit ScratchLease(SharedScratch& s) : s_(s), lock_(s.mu) {}
  ScratchLease(const ScratchLease&) = delete;
  ScratchLease& operator=(const ScratchLease&) = delete;
  // at least `bytes` of scratch, ordered after its previous use on stream st
  int acquire(size_t bytes, cudaStream_t st) {
    if (s_.buf.bytes < bytes || !s_.buf.p) {
      int rc = s_.order.wait_host();  // the old buffer may still be in use
      if (rc != 0) return rc;
      rc = s_.buf.reserve(bytes);
      if (rc != 0) return rc;
    }
    return s_.order.enter(st);
  }
  // record the end of this call's use on st (call after the last launch)
  int release(cudaStream_t st) { return s_.order.leave(st); }
  void* ptr() const { return s_.buf.p; }

 private:
  SharedScratch& s_;
  std::lock_guard<std::mutex> lock_;
};

// Per right-hand-side solver state, resident on the device.
struct RhsState {
  double rr;       // |r|^2 of the iterated residual
  double bb;       // |b|^2
  double rho2bb;   // stop threshold rho^2 |b|^2
  double alpha, beta;
  double sigma;    // stored sloppy p and Ap are p / sigma, Ap / sigma
  double c_r, c_p; // p_new / sigma_new = c_r r + c_p (p_old / sigma_old)
  double r_max2;   // largest |r|^2 since the last residual replacement
  double true_rr;  // |r_true|^2 at the last replacement
  double delta2;   // replacement trigger: |r|^2 < delta^2 r_max2
  int iter, max_iter;
  int active;      // 1 while iterating
  int need_ru;     // residual replacement requested
  int status;      // see SolveStatus
  int n_ru, restarts, restart_p;
};

enum SolveStatus { ST_RUNNING = 0, ST_ITER_CONV = 1, ST_MAXITER = 2, ST_DONE = 3, ST_FAILED = 4, ST_BREAKDOWN = 5 };

struct SolverWorkspace;    // solver.cu
struct ContractWorkspace;  // contract.cu
struct SolverWsDeleter {
  void operator()(SolverWorkspace* w) const;  // solver.cu
};
struct ContractWsDeleter {
  void operator()(ContractWorkspace* w) const;  // contract.cu
};
struct GradWorkspace;  // grad.cu
struct GradWsDeleter {
  void operator()(GradWorkspace* w) const;  // grad.cu
};
struct EoWorkspace;  // eo.cu
struct EoWsDeleter {
  void operator()(EoWorkspace* w) const;  // eo.cu
};

}  // namespace tsm

struct tsm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;  // blocking stream used when the caller passes NULL
  int sm_count = 0;
};

struct tsm_gauge {
  tsm_ctx* ctx = nullptr;
  tsm::Geom geom{};
  unsigned precisions = 0;
  tsm::DevBuf links[5];  // indexed by precision (TSM_DS: float-float twin of the FP64 copy)
  std::mutex mu;  // guards the caches below
  // workspaces keyed by solver kind + 64 * slot; slot 1 serves the TSM
  // driver's second stream, so two solves of one kind can run at once
  std::map<long long, std::unique_ptr<tsm::SolverWorkspace, tsm::SolverWsDeleter>> solver_ws;
  std::map<long long, std::unique_ptr<tsm::EoWorkspace, tsm::EoWsDeleter>> eo_ws;
  std::unique_ptr<tsm::ContractWorkspace, tsm::ContractWsDeleter> contract_ws[2];
  bool gamma_ready = false;  // insertion table uploaded (guarded by mu)
  tsm::SharedScratch tmp;     // operator scratch (M^dag M intermediate)
  tsm::SharedScratch eo_tmp;  // Schur operator scratch (three half-volume fields)
  std::mutex tsm_mu;       // guards the TSM buffers
  tsm::DevBuf tsm_acc;     // TSM accumulators and estimate
  tsm::DevBuf tsm_sol;     // solutions of one batch
  tsm::DevBuf tsm_sol2;    // the same for the second stream
  cudaStream_t aux_stream = nullptr;   // the TSM driver's second stream
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};  // fork and join events
  std::mutex grad_mu;      // guards grad_ws
  std::unique_ptr<tsm::GradWorkspace, tsm::GradWsDeleter> grad_ws;
  std::mutex tune_mu;      // guards nr_cache
  std::map<long long, int> nr_cache;  // autotuned right-hand sides per thread
  ~tsm_gauge();
};

namespace tsm {

inline cudaStream_t pick_stream(const tsm_gauge* g, void* s) {
  return s ? reinterpret_cast<cudaStream_t>(s) : g->ctx->stream;
}
inline bool has_prec(const tsm_gauge* g, int p) { return (g->precisions >> p) & 1u; }

// ---- launchers (dslash.cu)
// Right-hand sides per thread for the stencil on (field precision pin, link
// precision pl, nrhs), chosen by timing the candidates once per gauge.
int tuned_nr(tsm_gauge* g, int pin, int pl, int nrhs, cudaStream_t s, int* nr);
int dslash_apply(tsm_gauge* g, int prec, int op, double kappa, double mu, const void* in, void* out, int nrhs,
                 cudaStream_t s);
// out = op in with the link copy `prec_links` (may differ from the field precision `prec_field` only in
// the combinations instantiated there); gamma5 != 0 stores g5 * result.
int dslash_apply_mixed(tsm_gauge* g, int prec_field, int prec_links, int op, double kappa, double mu,
                       const void* in, void* out, int nrhs, int gamma5, cudaStream_t s);
// out = (c0 + i c1 g5) center + (h0 + i h1 g5) H in on full-volume F64/F32 fields (center may be null),
// H the hopping term of M = A0 - kappa H
int hop_general(tsm_gauge* g, int prec, const void* in, const void* center, void* out, int nrhs, double c0,
                double c1, double h0, double h1, cudaStream_t s);
// M or A on F64/F32 fields with a fixed number of right-hand sides per thread (no autotuning, no allocation).
int dslash_apply_fixed(tsm_gauge* g, int prec, int op, double kappa, double mu, const void* in, void* out, int nrhs,
                       int gamma5, int nr, cudaStream_t s);

// ---- fields (fields.cu)
int make_sources(const tsm_gauge* g, uint64_t seed, uint64_t first, int nsrc, int prec, void* out, cudaStream_t s);
// make_sources split by parity for the even-odd solvers (all extents even):
// even and odd halves, and diag_even = (cr + i ci g5) applied to the even half
int make_sources_eo(const tsm_gauge* g, uint64_t seed, uint64_t first, int nsrc, int prec, void* even, void* odd,
                    void* diag_even, double cr, double ci, cudaStream_t s);
// n_t fields: the source `source_id` kept on timeslices t_first .. t_first + n_t - 1, one each
int make_diluted_sources(const tsm_gauge* g, uint64_t seed, uint64_t source_id, int t_first, int n_t, int prec,
                         void* out, cudaStream_t s);
int spinor_pack(const tsm_gauge* g, int prec, const double* plain, void* native, int nrhs, double scale,
                cudaStream_t s);
int spinor_unpack(const tsm_gauge* g, int prec, const void* native, double* plain, int nrhs, double scale,
                  cudaStream_t s);
// dst(prec_dst) = a * src(prec_src) (+ g5 if gamma5), nrhs fields
int spinor_convert(const tsm_gauge* g, int prec_dst, void* dst, int prec_src, const void* src, int nrhs,
                   int gamma5, cudaStream_t s);
int build_links(tsm_gauge* g, const double* links_host);

// Host synthetic gauge field U = exp(i eps H) (fields.cu; host only)
int generate_gauge_host(const int dims[4], double eps, uint64_t seed, double* out);

// ---- solver (solver.cu)
// Solve M(mu) x = eta for nrhs right-hand sides.  eta (device, native layout of
// eta_prec) or, when eta is null, the Z4 sources (seed, first .. first+nrhs-1).
// gamma5_io != 0 multiplies eta by g5 on input and x by g5 on output.
// `slot` selects one of two workspace sets, so that solves on two streams can
// run at once (0 for every public entry point).
int solve_batch_impl(tsm_gauge* g, double kappa, double mu, int solver, double rho, int max_iter, int nrhs,
                     const void* eta, int eta_prec, uint64_t seed, uint64_t first, int out_prec, void* x_out,
                     int gamma5_io, tsm_solve_stats* stats, cudaStream_t s, int slot = 0);
int solver_precise_prec(int solver);
// Workspace, autotuned launch shapes (full-lattice solvers) and iteration-chunk
// graph of a later solve of nrhs right-hand sides at (kappa, mu) on `slot`, so
// that the solve itself allocates, times and captures nothing (solver.cu, eo.cu)
int prepare_solve(tsm_gauge* g, int solver, int nrhs, double kappa, double mu, int slot, cudaStream_t s);
int prepare_eo(tsm_gauge* g, int solver, int nrhs, double kappa, double mu, int slot, cudaStream_t s);
// The same with the even-odd preconditioned CG (solver carries TSM_SOLVER_EO; eo.cu).
int solve_batch_eo(tsm_gauge* g, double kappa, double mu, int solver, double rho, int max_iter, int nrhs,
                   const void* eta, int eta_prec, uint64_t seed, uint64_t first, int out_prec, void* x_out,
                   int gamma5_io, tsm_solve_stats* stats, cudaStream_t s, int slot);
// out = Mhat in (dag: Mhat^dag) on the odd sites of full-layout fields, zero on
// the even sites (eo.cu)
int schur_apply(tsm_gauge* g, int prec, int dag, double kappa, double mu, const void* in, void* out, int nrhs,
                cudaStream_t s);
// even-odd forms need every extent even: then every hop joins sites of
// opposite parity (x + y + z + t), and site i has checkerboard index i >> 1
inline bool eo_lattice(const Geom& g) { return !(g.L[0] % 2 || g.L[1] % 2 || g.L[2] % 2 || g.L[3] % 2); }
// solver kind without flags; -1 if unknown
inline int solver_kind(int solver) {
  const int k = solver & ~TSM_SOLVER_EO;
  return (k >= TSM_SOLVER_F64 && k <= TSM_SOLVER_LP_BF16) ? k : -1;
}
int solve_batch_multi(tsm_batch_item* items, int n, int solver, double rho, int max_iter, cudaStream_t s);
int solver_output_prec(int solver);
unsigned solver_link_precs(int solver);

// ---- contraction (contract.cu)
int contract_loops(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                   const int* mom_host, double* out_dev, int accumulate, cudaStream_t s, int slot = 0);
// Workspace, insertion table and tuned operator shape of a later contract_loops of nsrc sources on `slot`
int prepare_contract(tsm_gauge* g, int prec, int nsrc, int n_mom, const int* mom_host, int slot, cudaStream_t s);
// Standard-estimator loops of sources eta (time-diluted: t0[r] >= 0, or volume
// sources: t0[r] = -1) and their solutions s (contract.cu)
int contract_tdil(tsm_gauge* g, int prec, const void* s_dev, const void* eta_dev, int nsrc, const int* t0_host,
                  int n_mom, const int* mom_host, double* out_dev, int accumulate, cudaStream_t s);
// Standard-estimator loops with the hopping parameter expansion of the 16
// ultra-local insertions (both flavours); derivative insertions plain
int contract_hpe(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, const void* eta_dev, int nsrc,
                 const int* t0_host, int n_mom, const int* mom_host, double* out_dev, int accumulate, cudaStream_t s);
int contract_loops_noalloc(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                           const int* mom_host, double* out_dev, int accumulate, cudaStream_t s);

// ---- loop backward (grad.cu)
int loops_backward(tsm_gauge* g, double kappa, double mu, int prec, const void* s_dev, int nsrc, int n_mom,
                   const int* mom, const double* grad_dev, int solver, double rho, int max_iter, double* dmu_host,
                   void* grad_eta_dev, cudaStream_t s);

// ---- misc
int momentum_table(int p2max, std::vector<int>& out);

// ---- profiling (prof.cu)
bool profiling();
void count_launches(long long n);  // kernels enqueued by the library (graph nodes included)
void prof_add(const char* name, double seconds, double bytes, double flops);
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  int begin(cudaStream_t s);
  int end(cudaStream_t s);
  double seconds();  // waits for the end event
  ~EventPair();
};
inline double spinor_site_bytes(int prec) { return 16.0 * spinor_chunks(prec); }
inline double link_site_bytes(int prec) { return (double)link_bytes(prec, 1); }

}  // namespace tsm
