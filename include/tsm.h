/*
 * tsm.h -- C ABI of the GB300 (sm_103a) library for disconnected fermion
 * loops with twisted-mass Wilson fermions and the Truncated Solver Method,
 * after A. Vaquero et al., "A QUDA-branch to compute disconnected diagrams
 * in GPUs" (arXiv:1401.6750).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice: dims = {Lx, Ly, Lz, T}; site index i = x + Lx*(y + Ly*(z + Lz*t));
 *   V = Lx*Ly*Lz*T.  Direction mu = 0,1,2,3 means x, y, z, t.
 * Links (host input): complex128 U_mu(x)_{ab} at
 *   links[((i*4 + mu)*3 + a)*3 + b] as {re, im} double pairs, i.e. the
 *   row-major array [V][4][3][3][2].  The matrices must be SU(3) (the 16- and
 *   32-bit copies keep two rows and rebuild the third).
 * Boundary: periodic in space; the link U_t on the last timeslice carries
 *   the factor t_bc (+1 periodic, -1 antiperiodic), in the Dirac operator and
 *   in the derivative insertions alike.
 * Operator (Eq. 1 solves M s = eta; the paper does not print M, this is the
 *   standard kappa-normalised twisted-mass Wilson form, u flavour):
 *     M = A + i mu' g5,   mu' = 2 kappa mu,
 *     A psi(x) = psi(x) - kappa sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
 *                                      + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ],
 *     M^dag = g5 M(-mu) g5.
 *   Gamma matrices: chiral basis, g_k = [[0, -i s_k], [i s_k, 0]] (k = x, y, z
 *   with Pauli s_k), g_t = [[0, 1], [1, 0]], g5 = g_x g_y g_z g_t = diag(1,1,-1,-1).
 * Spinor fields on the device use a "chunked" layout per precision: the 12
 *   complex components c = 3*spin + colour of one site are cut into 16-byte
 *   chunks, and chunk j of all sites is contiguous:
 *     byte offset of chunk j, site i, right-hand side r = ((r*NCH + j)*V + i)*16
 *   F64: NCH = 12, chunk j = component j as {re, im} doubles;
 *   F32: NCH = 6,  chunk j = components 2j, 2j+1 as 4 floats;
 *   F16 / BF16: NCH = 3, chunk j = components 4j .. 4j+3 as 8 halves.
 *   tsm_spinor_pack / tsm_spinor_unpack convert from / to the plain layout
 *   [nrhs][V][4][3][2] of doubles.
 *
 * Ownership: the library owns contexts, gauge handles and its workspaces.
 *   Caller pointers are only used during the call (and the work it enqueues
 *   on the caller's stream); nothing is freed or retained.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = the context's
 *   own blocking stream, ordered with the legacy default stream).  Calls that
 *   return host data synchronise that stream.
 * Threads: calls on one handle may come from several host threads and
 *   streams.  The library's per-handle workspaces and scratch are guarded on
 *   the host, and each one's use on the GPU is ordered across streams by an
 *   event (a stream that takes it over waits for the previous user's last
 *   launch).  Apart from tsm_create_gauge and tsm_destroy_gauge, which
 *   synchronise the device, the library enqueues nothing on the legacy
 *   default stream, so its calls do not invalidate a graph capture on another
 *   thread's blocking stream.  Inside a capture the cross-stream event waits
 *   are left out: captured calls on one handle must be ordered by the
 *   caller.
 * Errors: every int-returning call returns TSM_OK (0) or a TSM_ERR_* code;
 *   tsm_last_error() gives a message for the calling thread.  No exception
 *   crosses the ABI.  A call that fails with TSM_ERR_INVALID_ARG has not
 *   touched the device.
 */
#ifndef TSM_H
#define TSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum tsm_status {
  TSM_OK = 0,
  TSM_ERR_INVALID_ARG = 1,
  TSM_ERR_CUDA = 2,
  TSM_ERR_OOM = 3,
  TSM_ERR_NOT_CONVERGED = 4, /* outputs are still written; see the stats */
  TSM_ERR_NONFINITE = 5,     /* NaN/Inf met in an input or a residual */
  TSM_ERR_UNIMPLEMENTED = 6
};

enum tsm_prec { TSM_F64 = 0, TSM_F32 = 1, TSM_F16 = 2, TSM_BF16 = 3 };
#define TSM_PREC_BIT(p) (1u << (p))

enum tsm_op {
  TSM_OP_M = 0,     /* M(mu)                                  */
  TSM_OP_MDAG = 1,  /* M(mu)^dag                              */
  TSM_OP_A = 2,     /* Wilson part A = M(mu = 0)              */
  TSM_OP_MDAGM = 3, /* M^dag M                                */
  /* Even-odd Schur operator Mhat = M_oo - M_oe M_ee^{-1} M_eo and its adjoint
   * (see TSM_SOLVER_EO): they act on the odd sites of the input and write the
   * result on the odd sites, zeros on the even sites.  Need every extent
   * even. */
  TSM_OP_MHAT = 4,
  TSM_OP_MHATDAG = 5
};

/* Solvers for Eq. 1 (all CG on M^dag M, x0 = 0, see tsm_solve_sources). */
enum tsm_solver {
  TSM_SOLVER_F64 = 0,          /* FP64 links and vectors throughout             */
  TSM_SOLVER_F32_RELIABLE = 1, /* FP32 CG; true residual and solution sum in     *
                                * float-float (about 44 significant bits), for  *
                                * rho down to about 1e-9 (HP); tighter: F64     */
  TSM_SOLVER_LP_F16 = 2,       /* FP16 links/p/Ap, FP32 x and r (LP)            */
  TSM_SOLVER_LP_BF16 = 3,      /* BF16 links/p/Ap, FP32 x and r (LP)            */
  /* Flag OR-ed into any of the above: solve the even-odd (Schur complement)
   * system Mhat s_o = eta_o - M_oe M_ee^{-1} eta_e by CG on Mhat^dag Mhat on the
   * odd sites, then reconstruct s_e = M_ee^{-1}(eta_e - M_eo s_o).  Same
   * solutions and output layout; needs every extent even.  `rho` then bounds the
   * residual of the preconditioned normal equations, and the stats report
   * it.  Not available in tsm_solve_batch. */
  TSM_SOLVER_EO = 16
};

#define TSM_N_INSERTIONS 160

typedef struct tsm_ctx tsm_ctx;
typedef struct tsm_gauge tsm_gauge;

/* Per right-hand side solve record. */
typedef struct {
  int iterations;       /* CG iterations (sloppy operator applications / 2)  */
  int reliable_updates; /* residual replacements                           */
  int converged;        /* 1 if the true residual met rho                   */
  int restarts;         /* restarts after a failed true-residual check      */
  double true_residual; /* |M^dag eta - M^dag M x| / |M^dag eta|, precise op */
} tsm_solve_stats;

/* ------------------------------------------------------------------ setup */

/* Bind a context to CUDA device `device` (it becomes current on this host
 * thread).  Returns TSM_ERR_CUDA if the device is unusable or not sm_103. */
int tsm_ctx_create(int device, tsm_ctx** out);
void tsm_ctx_destroy(tsm_ctx* ctx);

/* Upload a gauge field (layout above) and build the device copies named in
 * `precisions` (bitmask of TSM_PREC_BIT(TSM_F64 | ...)).  FP64 keeps all 18
 * reals per link; FP32/FP16/BF16 keep the first two rows (12 reals) and
 * rebuild row 3 = conj(row1 x row2) on use.  Each Lx..T must be >= 2.  The
 * host array is only read during the call. */
int tsm_create_gauge(tsm_ctx* ctx, const int dims[4], const double* links_host,
                     int t_bc, unsigned precisions, tsm_gauge** out);
void tsm_destroy_gauge(tsm_gauge* g);

/* Bytes of a native spinor field of `nrhs` right-hand sides. */
size_t tsm_spinor_bytes(const tsm_gauge* g, int prec, int nrhs);

/* plain [nrhs][V][4][3][2] doubles (device) -> native layout of `prec`,
 * multiplying by `scale` before rounding.  Values beyond the range of the
 * target type become +-Inf (the caller chooses `scale`). */
int tsm_spinor_pack(const tsm_gauge* g, int prec, const double* plain_dev,
                    void* native_dev, int nrhs, double scale, void* stream);
/* native -> plain doubles, multiplying by `scale` after widening. */
int tsm_spinor_unpack(const tsm_gauge* g, int prec, const void* native_dev,
                      double* plain_dev, int nrhs, double scale, void* stream);

/* ----------------------------------------------------------- hot path ops */

/* out = op(kappa, mu) in, for nrhs fields in native layout of `prec` (links
 * of the same precision must exist).  Eq. 1's M and its relatives; the sum
 * runs in FP32 for F32/F16/BF16 fields and FP64 for F64.  in and out must
 * not overlap. */
int tsm_dslash_tm(tsm_gauge* g, double kappa, double mu, int op, int prec,
                  const void* in_dev, void* out_dev, int nrhs, void* stream);

/* Z4 volume sources (Sec. 2 "random stochastic sources", generated on the
 * GPU as Sec. 2.4 proposes): component c = 3*spin + colour of site i of
 * source r = first_src + k takes bits 2c, 2c+1 of word 0 of
 * Philox4x64-10(counter = {i, 0, 0, 0}, key = {noise_seed, r}) and the value
 * i^bits.  Written in native layout of `prec`, nsrc fields. */
int tsm_make_sources(tsm_gauge* g, uint64_t noise_seed, uint64_t first_src,
                     int nsrc, int prec, void* out_dev, void* stream);

/* Synthetic gauge field on the host (no GPU use): U_mu(x) = exp(i eps H),
 * H = sum_a h_a lambda_a / 2 with h_a ~ N(0, 1) and lambda_a the Gell-Mann
 * matrices, the stand-in for the paper's ensembles.  The eight normals of
 * link (site i, direction mu) are Box-Muller pairs of the eight 32-bit
 * halves (low half first, u = (w + 1/2) / 2^32) of the words of
 * Philox4x64-10(counter = {4 i + mu, 0, 0, 0}, key = {seed, 0x67617567});
 * the exponential goes through the eigenvectors of H (Jacobi rotations), in
 * FP64.  links_out: [V][4][3][3] complex as 18 doubles per link, row-major,
 * site i = x + Lx*(y + Ly*(z + Lz*t)) -- the layout tsm_create_gauge takes. */
int tsm_generate_gauge_host(const int dims[4], double eps, uint64_t seed,
                            double* links_out);

/* Time dilution (Sec. 2.2): n_t fields, field k being the Z4 source of
 * (noise_seed, source_id) -- the same values tsm_make_sources gives for
 * first_src = source_id -- kept on timeslice t_first + k and zero on every
 * other timeslice, so the T diluted sources of one noise vector sum to the
 * volume source.  Needs 0 <= t_first and t_first + n_t <= T.  Written in
 * native layout of `prec` (F64, F32, F16 or BF16). */
int tsm_make_diluted_sources(tsm_gauge* g, uint64_t noise_seed,
                             uint64_t source_id, int t_first, int n_t,
                             int prec, void* out_dev, void* stream);

/* Solve M s_r = eta_r (Eq. 1) for the Z4 sources r = first_src ..
 * first_src + nsrc - 1 by CG on M^dag M with x0 = 0, stopping when the
 * iterated residual of the normal equations drops below rho (1 - c) and the
 * true residual (recomputed with the precise operator: FP64 for F64,
 * float-float for F32_RELIABLE, FP32 for the LP solvers) confirms it;
 * otherwise the iteration restarts from the true residual, up to max_iter in
 * total.  c is a margin for the precise operator's own rounding (1e-6 FP64,
 * 1e-2 float-float, 1e-3 FP32), so that the true residual of each returned
 * solution, recomputed exactly, is at most rho.
 * Solutions are written in native layout: F64 for TSM_SOLVER_F64 and
 * TSM_SOLVER_F32_RELIABLE (its float-float accumulated solution), F32 for the LP
 * solvers.  stats_host (optional) receives nsrc records.  Returns
 * TSM_ERR_NOT_CONVERGED if any source missed rho (outputs still written).
 * Right-hand sides are batched `nrhs_per_launch` at a time (<= 0: all). */
int tsm_solve_sources(tsm_gauge* g, double kappa, double mu, int solver,
                      double rho, int max_iter, uint64_t noise_seed,
                      uint64_t first_src, int nsrc, int nrhs_per_launch,
                      void* s_dev, tsm_solve_stats* stats_host, void* stream);

/* One instance of an uneven batch: its own gauge field (lattice), twisted
 * mass and Z4 sources r = first_src .. first_src + nsrc - 1. */
typedef struct {
  tsm_gauge* gauge;
  double kappa, mu;
  uint64_t noise_seed, first_src;
  int nsrc;
  void* s_dev;                  /* out: nsrc solutions, native, solver output precision */
  tsm_solve_stats* stats_host;  /* optional: nsrc records */
} tsm_batch_item;

/* Solve every instance of an uneven batch together: each CG kernel is ONE
 * launch over all instances (lattices of different sizes, different twisted
 * masses), with a convergence flag per right-hand side; an instance is done
 * when all its right-hand sides are.  Same solvers, stopping rule and
 * results as tsm_solve_sources on each instance alone.  All gauges must live
 * in contexts of the same device.  Allocates its workspace per call. */
int tsm_solve_batch(tsm_batch_item* items, int n_items, int solver, double rho,
                    int max_iter, void* stream);

/* Solve op x = b for caller right-hand sides, op = TSM_OP_M (M x = b) or
 * TSM_OP_MDAG (M^dag x = b, through M^dag = g5 M(-mu) g5).  b and x in the
 * native layout of the solver's output precision (F64 for TSM_SOLVER_F64 and
 * TSM_SOLVER_F32_RELIABLE, F32 for the LP solvers).  Same stopping rule as
 * tsm_solve_sources. */
int tsm_invert(tsm_gauge* g, double kappa, double mu, int op, int solver,
               double rho, int max_iter, const void* b_dev, void* x_dev,
               int nrhs, tsm_solve_stats* stats_host, void* stream);

/* One-end-trick loops (Sec. 2.1.1, Sec. 2.2) of nsrc solved sources s
 * (native layout, prec F64 or F32), summed over the sources:
 *   ins = 80 f + g             ultra-local Gamma_g
 *   ins = 80 f + 16 + 16 mu + g  one-derivative, direction mu
 * f = 0: with tau_3,  -2 i mu' s^dag g5 X s        (estimates Tr[X(G_u - G_d)])
 * f = 1: without,      2      s^dag g5 X g5 A s    (estimates Tr[X(G_u + G_d)])
 * Gamma_g = g_x^{b0} g_y^{b1} g_z^{b2} g_t^{b3} (b_j = bit j of g);
 * derivative X = 1/4 [psibar(x) G U(x) psi(x+mu) - psibar(x+mu) G U(x)^dag psi(x)
 *                   + psibar(x-mu) G U(x-mu) psi(x) - psibar(x) G U(x-mu)^dag psi(x-mu)],
 * each projected per timeslice onto the momenta mom[k] = {nx, ny, nz}:
 *   L(k, t) = sum_xyz L(x, t) exp(-2 pi i (nx x/Lx + ny y/Ly + nz z/Lz)).
 * out_dev: device doubles [160][n_mom][T][2]; with accumulate != 0 the sums
 * are added to out_dev, otherwise out_dev is overwritten.  |n_i| <= 8. */
int tsm_contract_loops(tsm_gauge* g, double kappa, double mu, int prec,
                       const void* s_dev, int nsrc, int n_mom, const int* mom,
                       double* out_dev, int accumulate, void* stream);

/* Backward of the loops for automatic differentiation (used by the PyTorch
 * autograd wrapper; the derivatives of Sec. 2.1.1's loops with respect to
 * the twisted mass and the sources, by the adjoint method through Eq. 1).
 * Given the solutions s_r = M(mu)^{-1} eta_r (native, prec F64 or F32, nsrc
 * fields) used to form the loops L = sum_r [tsm_contract_loops of s_r] on the
 * momenta mom, and grad_dev = dl/dRe L + i dl/dIm L for a real loss l
 * (device doubles [160][n_mom][T][2]), this computes
 *   *dmu_host   = dl/dmu   (through s and the explicit mu' of the tau_3 loops)
 *   grad_eta_dev (optional, native prec, nsrc fields) = dl/dRe eta + i dl/dIm eta
 * with one adjoint solve lambda_r = M^{-dag} g_r per source, by `solver`
 * (TSM_SOLVER_F64 or TSM_SOLVER_F32_RELIABLE) to `rho`.  Synchronises. */
int tsm_loops_backward(tsm_gauge* g, double kappa, double mu, int prec,
                       const void* s_dev, int nsrc, int n_mom, const int* mom,
                       const double* grad_dev, int solver, double rho,
                       int max_iter, double* dmu_host, void* grad_eta_dev,
                       void* stream);

/* Loops of the 160 insertions from the standard estimator, for sources that
 * are time-diluted (the paper's single-timeslice contraction, Sec. 2.2) or
 * not: for nsrc sources eta_r and their solutions s_r = M(mu)^{-1} eta_r
 * (both native F64 or F32 fields, nsrc each), the bilinear
 * psibar(y) K psi(z) -> Tr[K G(z, y)] is estimated by eta(y)^dag K s(z) for
 * the u flavour and, through g5-hermiticity (G_d = g5 G_u^dag g5), by
 * conj(eta(z)^dag g5 K^dag g5 s(y)) for the d flavour; insertion f*80 + i
 * carries u - d (f = 0, with tau_3) or u + d (f = 1), with the insertion
 * index, derivative form and layout [160][n_mom][T][2] of tsm_contract_loops,
 * summed (not averaged) over the sources.  t0_host (optional, nsrc values)
 * gives each source's timeslice, or -1 for a volume source; only the
 * timeslices a source touches are contracted (t0, and t0 - 1 for the time
 * derivative).  Both flavour combinations are formed per site before the
 * Fourier sums.  accumulate != 0 adds to out_dev.  Asynchronous on
 * `stream`. */
int tsm_contract_tdil(tsm_gauge* g, int prec, const void* s_dev,
                      const void* eta_dev, int nsrc, const int* t0_host,
                      int n_mom, const int* mom, double* out_dev,
                      int accumulate, void* stream);

/* tsm_contract_tdil with the hopping parameter expansion (HPE, Sec. 2.3)
 * for the 16 ultra-local insertions of both flavours: with M = A0 - kappa H
 * (A0 = 1 + i mu' g5) and Y = A0^{-1} kappa H, G = sum_{k<4} Y^k A0^{-1} +
 * Y^4 G; the exact diagonal of the first four terms (a constant per site,
 * orders 0 and 2, computed in closed form) is added at p = 0 once per
 * source on the timeslices it covers, and the remainder is estimated by
 * eta^dag X (Y^4 s).  The derivative insertions are those of
 * tsm_contract_tdil.  kappa, mu must be those of the solves; needs every
 * extent >= 4 (shorter extents close paths of length < 4 around the
 * lattice).  Same arguments and layout otherwise. */
int tsm_contract_hpe(tsm_gauge* g, double kappa, double mu, int prec,
                     const void* s_dev, const void* eta_dev, int nsrc,
                     const int* t0_host, int n_mom, const int* mom,
                     double* out_dev, int accumulate, void* stream);

/* Allocation-free variant of tsm_contract_loops (the paper has no
 * counterpart: it is an interface convenience).  It is meant for callers
 * that cannot call cudaMalloc during the call -- e.g. code running under a
 * memory pool or allocator that forbids new device allocations, or latency-
 * sensitive loops where an allocation would synchronise the device.  The
 * caller still passes the solutions and the output; the library's own
 * scratch (g5 A s for every source, the 160 site fields, the per-plane
 * partial projections and a copy of the momentum list) lives in a fixed
 * array of TSM_CONTRACT_NOALLOC_MAX_BYTES compiled into the library, which
 * every GPU that loads the library holds until the process exits.  Needs
 *   256-rounded(12 n_mom) + 256-rounded(nsrc * V * 16 * NCH)
 *   + 256-rounded(160 * V * c) + 256-rounded(Lz * T * 160 * (2R+1)^2 * c)
 *   bytes (R = max |n_i|; c = 8 for F32 solutions, 16 for F64)
 * and returns TSM_ERR_INVALID_ARG, touching nothing, when that exceeds the
 * maximum.  The first call on a device looks up the array's device address
 * and uploads a constant table there (make it before any stream capture);
 * no call allocates device memory.  Every call copies the momentum list from
 * the caller's host array, so calls inside a stream capture are not
 * supported (a graph would re-read that host array at each replay).  That address is kept for the life of the
 * process: a cudaDeviceReset after the first call is not supported.  All calls share the array and it keeps
 * the last call's contents: calls that overlap on the GPU (two streams, two
 * threads) race.  Results equal tsm_contract_loops'. */
#define TSM_CONTRACT_NOALLOC_MAX_BYTES (32 * 1024 * 1024)
int tsm_contract_loops_noalloc(tsm_gauge* g, double kappa, double mu, int prec,
                               const void* s_dev, int nsrc, int n_mom,
                               const int* mom, double* out_dev, int accumulate,
                               void* stream);

typedef struct {
  double kappa, mu;
  int n_lp, n_hp;          /* low-precision (bulk) and correction source counts */
  double rho_lp, rho_hp;   /* stopping residuals (Sec. 2.1: ~1e-2 and ~1e-8)    */
  int lp_solver, hp_solver;/* tsm_solver values                                 */
  uint64_t noise_seed;     /* bulk sources 0..n_lp-1, corrections n_lp..+n_hp-1 */
  int max_iter;
  int nrhs_per_launch;     /* right-hand sides per batched solve (<= 0: 12)     */
  int n_mom;
  const int* mom;          /* host [n_mom][3]                                    */
} tsm_params;

typedef struct {
  int lp_iterations_total, hp_iterations_total;
  int lp_max_iterations, hp_max_iterations;
  double lp_max_true_residual, hp_max_true_residual;
  int n_not_converged;
  double seconds;
} tsm_stats;

/* Truncated Solver Method estimate (Sec. 2.1):
 *   E = (1/N_LP) sum_bulk L_LP + (1/N_HP) sum_corr [L_HP - L_LP]
 * (the correction term is dropped when n_hp = 0), with L the tsm_contract_loops
 * sums of single sources.  loops_host: [160][n_mom][T][2] doubles.
 * parts_host (optional): the three source-summed accumulators
 * [3][160][n_mom][T][2] in the order bulk-LP, corr-HP, corr-LP.  Synchronises
 * `stream`.
 * Concurrency: when n_hp > 0 the correction sources' HP and LP solves run from
 * a library worker thread on a second stream that the gauge handle owns,
 * created at the device's highest stream priority, beside the bulk solves on
 * `stream`; the call returns after both, with `stream` ordered after the
 * second stream's work.  TSM_STREAMS=1 in the environment runs everything on
 * `stream` from the calling thread. */
int tsm_solve_tsm(tsm_gauge* g, const tsm_params* p, double* loops_host,
                  double* parts_host, tsm_stats* stats, void* stream);

/* As tsm_solve_tsm, with the estimate written to device memory loops_dev
 * ([160][n_mom][T][2] doubles) and, if parts_dev is not NULL, the three
 * accumulators to parts_dev ([3][160][n_mom][T][2]); nothing is copied to
 * the host.  stats (optional) forces a synchronisation of `stream`. */
int tsm_solve_tsm_dev(tsm_gauge* g, const tsm_params* p, double* loops_dev,
                      double* parts_dev, tsm_stats* stats, void* stream);

/* ---------------------------------------------------------------- helpers */

/* Binary-weight storage of loop sums (Sec. 2.1.1, Fig. 2).  The file of
 * weight 2^k, "<path_prefix>.w<2^k>.bin", holds the sum of the contractions
 * of the 2^k sources 2^k - 1 .. 2^{k+1} - 2 (0-based ids; the paper's
 * File.1, File.2, File.4 ... counting from 1), n_values doubles after a
 * header with an FNV-1a checksum.  Any N sources are recovered from the files
 * of N's set bits, so N sources take log2 N files.  Host-only calls (no GPU
 * use) except tsm_accumulate_blocks.
 *   tsm_binstore_open   opens (the directory must exist) and validates every
 *                       block file present; TSM_ERR_INVALID_ARG on a corrupt,
 *                       truncated or mismatched file.  Free with _close.
 *   tsm_binstore_sources  2^K - 1 for the contiguous blocks 0..K-1 present:
 *                       where an interrupted accumulation resumes.
 *   tsm_binstore_block  the source range of block k.
 *   tsm_binstore_put    writes block k (written to a temporary name, then
 *                       renamed into place).
 *   tsm_binstore_mean   out = (sum of the blocks of n's bits) / n; fails if
 *                       one of them is missing.
 *   tsm_accumulate_blocks  computes the bulk LP loops (p's lp_solver, rho_lp,
 *                       kappa, mu, noise_seed, max_iter, nrhs_per_launch,
 *                       momenta; one-end contraction as tsm_solve_tsm) of
 *                       every block from the first one missing up to
 *                       k_end - 1 and stores them; the store's n_values must
 *                       be 160 * n_mom * T * 2.  stats: LP fields only. */
typedef struct tsm_binstore tsm_binstore;
int tsm_binstore_open(const char* path_prefix, size_t n_values,
                      tsm_binstore** out);
void tsm_binstore_close(tsm_binstore* st);
long long tsm_binstore_sources(const tsm_binstore* st);
int tsm_binstore_block(int k, long long* first_source, long long* n_sources);
int tsm_binstore_put(tsm_binstore* st, int k, const double* block_sum_host);
int tsm_binstore_mean(const tsm_binstore* st, long long n, double* out_host);
int tsm_accumulate_blocks(tsm_gauge* g, const tsm_params* p, tsm_binstore* st,
                          int k_end, tsm_stats* stats, void* stream);

/* Momenta n with n^2 <= p2max, ordered by n^2 then lexicographically
 * (Sec. 2.3 cut on p^2); writes min(count, cap) triples, returns the count
 * (123 for p2max = 9), or -1 if p2max < 0. */
int tsm_momentum_table(int p2max, int* out, int cap);

/* Opt-in kernel timing.  While enabled, solver iterations run one at a time
 * without CUDA graphs and every kernel of the hot path is bracketed by CUDA
 * events on its stream; each launch adds its duration and its algorithmic
 * traffic (every operand read or written once; links once per launch) and
 * flop count to a per-kernel-class total.  Enabling clears the totals. */
typedef struct {
  char name[48];
  long long launches;
  double seconds; /* sum of event-timed launch durations */
  double bytes;   /* sum of algorithmic bytes              */
  double flops;   /* sum of algorithmic flops              */
} tsm_kernel_profile;
int tsm_profile_enable(int on);
/* Total kernels the library has enqueued in this process (kernel nodes of
 * replayed CUDA graphs included). */
long long tsm_kernel_launches(void);
/* Copies up to cap entries, returns the number of kernel classes. */
int tsm_profile_read(tsm_kernel_profile* out, int cap);

const char* tsm_strerror(int code);
const char* tsm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TSM_H */
