// Binary-weight storage of loop sums (Sec. 2.1.1, Fig. 2) and the block
// driver that fills it.
//
// The file of weight 2^k holds the sum of the contractions of the 2^k
// sources 2^k - 1 .. 2^{k+1} - 2 (0-based ids; the paper's File.1, File.2,
// File.4 ... counting sources from 1).  Any N sources are recovered from the
// files of N's set bits, so storing N sources takes log2 N files.  Blocks
// are written whole, to a temporary name renamed into place, with a header
// and an FNV-1a checksum; opening a store validates every file and counts
// the contiguous blocks 0 .. K-1 present (2^K - 1 sources), which is where
// an interrupted accumulation resumes.
#include <errno.h>
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace tsm {
namespace {

constexpr int kMaxBlocks = 40;
const char kMagic[8] = {'T', 'S', 'M', 'B', 'W', 'v', '1', '\0'};

struct BlockHeader {
  char magic[8];
  uint32_t header_bytes;
  uint32_t k;
  uint64_t first_source;
  uint64_t n_sources;
  uint64_t n_values;
  uint64_t checksum;  // FNV-1a 64 over the value bytes
};

uint64_t fnv1a(const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

std::string block_path(const std::string& prefix, int k) {
  char suffix[48];
  snprintf(suffix, sizeof(suffix), ".w%llu.bin", (unsigned long long)1 << k);
  return prefix + suffix;
}

}  // namespace
}  // namespace tsm

struct tsm_binstore {
  std::string prefix;
  size_t n_values = 0;
  bool present[tsm::kMaxBlocks] = {false};
};

namespace tsm {
namespace {

// Reads block k into `out` (n values) after validating it; TSM_OK, or an error
// code with the reason recorded.
int read_block(const tsm_binstore* st, int k, double* out) {
  const std::string path = block_path(st->prefix, k);
  FILE* f = fopen(path.c_str(), "rb");
  if (!f) return fail(TSM_ERR_INVALID_ARG, "block file %s: %s", path.c_str(), strerror(errno));
  BlockHeader h;
  const size_t got = fread(&h, 1, sizeof(h), f);
  int rc = TSM_OK;
  if (got != sizeof(h) || memcmp(h.magic, kMagic, 8) != 0 || h.header_bytes != sizeof(h))
    rc = fail(TSM_ERR_INVALID_ARG, "%s is not a block file", path.c_str());
  else if (h.k != (uint32_t)k || h.first_source != ((1ull << k) - 1) || h.n_sources != (1ull << k))
    rc = fail(TSM_ERR_INVALID_ARG, "%s holds block %u, expected %d", path.c_str(), h.k, k);
  else if (h.n_values != st->n_values)
    rc = fail(TSM_ERR_INVALID_ARG, "%s holds %llu values, expected %zu", path.c_str(),
              (unsigned long long)h.n_values, st->n_values);
  std::vector<double> tmp;
  if (rc == TSM_OK) {
    double* dst = out;
    if (!dst) {
      tmp.resize(st->n_values);
      dst = tmp.data();
    }
    if (fread(dst, sizeof(double), st->n_values, f) != st->n_values)
      rc = fail(TSM_ERR_INVALID_ARG, "%s is truncated", path.c_str());
    else if (fnv1a(dst, st->n_values * sizeof(double)) != h.checksum)
      rc = fail(TSM_ERR_INVALID_ARG, "%s fails its checksum", path.c_str());
  }
  fclose(f);
  return rc;
}

}  // namespace

// ---------------------------------------------------------------- block driver
// Bulk LP loops of the sources of blocks k0 .. k_end - 1, each block solved
// in batches of p->nrhs_per_launch, contracted into a device accumulator,
// copied out and written.
int accumulate_blocks(tsm_gauge* g, const tsm_params* p, tsm_binstore* st, int k_end, tsm_stats* stats,
                      cudaStream_t s) {
  const size_t n_out = (size_t)160 * p->n_mom * g->geom.L[3] * 2;
  if (n_out != st->n_values)
    return fail(TSM_ERR_INVALID_ARG, "store holds %zu values per block, these loops have %zu", st->n_values, n_out);
  const int batch = p->nrhs_per_launch > 0 ? std::min(p->nrhs_per_launch, 1024) : 12;
  const int op = (solver_kind(p->lp_solver) == TSM_SOLVER_F64) ? TSM_F64 : TSM_F32;
  DevBuf acc, sol;
  TSM_TRY(acc.reserve(sizeof(double) * n_out));
  std::vector<double> host(n_out);
  std::vector<tsm_solve_stats> ss(batch);
  int k0 = 0;
  while (k0 < kMaxBlocks && st->present[k0]) ++k0;
  long long iters = 0, iters_max = 0, not_conv = 0;
  double res_max = 0.0;
  for (int k = k0; k < k_end; ++k) {
    const long long first = (1ll << k) - 1, count = 1ll << k;
    TSM_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(double) * n_out, s));
    for (long long r0 = 0; r0 < count; r0 += batch) {
      const int nb = (int)std::min<long long>(batch, count - r0);
      TSM_TRY(sol.reserve(tsm_spinor_bytes(g, op, nb)));
      const int rc = solve_batch_impl(g, p->kappa, p->mu, p->lp_solver, p->rho_lp, p->max_iter, nb, nullptr, 0,
                                      p->noise_seed, (uint64_t)(first + r0), op, sol.p, 0, ss.data(), s);
      if (rc != TSM_OK && rc != TSM_ERR_NOT_CONVERGED) return rc;
      for (int j = 0; j < nb; ++j) {
        iters += ss[j].iterations;
        iters_max = std::max<long long>(iters_max, ss[j].iterations);
        res_max = std::max(res_max, ss[j].true_residual);
        not_conv += !ss[j].converged;
      }
      TSM_TRY(contract_loops(g, p->kappa, p->mu, op, sol.p, nb, p->n_mom, p->mom, acc.as<double>(), 1, s));
    }
    TSM_CUDA(cudaMemcpyAsync(host.data(), acc.p, sizeof(double) * n_out, cudaMemcpyDeviceToHost, s));
    TSM_CUDA(cudaStreamSynchronize(s));
    const int rc = tsm_binstore_put(st, k, host.data());
    if (rc != TSM_OK) return rc;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->lp_iterations_total = (int)iters;
    stats->lp_max_iterations = (int)iters_max;
    stats->lp_max_true_residual = res_max;
    stats->n_not_converged = (int)not_conv;
  }
  if (not_conv) return fail(TSM_ERR_NOT_CONVERGED, "%lld solves missed rho", not_conv);
  return TSM_OK;
}

}  // namespace tsm

using namespace tsm;

extern "C" {

int tsm_binstore_open(const char* path_prefix, size_t n_values, tsm_binstore** out) {
  if (!path_prefix || !*path_prefix || !out || n_values == 0)
    return fail(TSM_ERR_INVALID_ARG, "tsm_binstore_open: bad argument");
  *out = nullptr;
  tsm_binstore* st = new tsm_binstore();
  st->prefix = path_prefix;
  st->n_values = n_values;
  for (int k = 0; k < kMaxBlocks; ++k) {
    struct stat sb;
    if (stat(block_path(st->prefix, k).c_str(), &sb) != 0) continue;
    const int rc = read_block(st, k, nullptr);
    if (rc != TSM_OK) {
      delete st;
      return rc;
    }
    st->present[k] = true;
  }
  *out = st;
  return TSM_OK;
}

void tsm_binstore_close(tsm_binstore* st) { delete st; }

long long tsm_binstore_sources(const tsm_binstore* st) {
  if (!st) return -1;
  int k = 0;
  while (k < kMaxBlocks && st->present[k]) ++k;
  return (1ll << k) - 1;
}

int tsm_binstore_block(int k, long long* first_source, long long* n_sources) {
  if (k < 0 || k >= kMaxBlocks) return fail(TSM_ERR_INVALID_ARG, "block %d out of range", k);
  if (first_source) *first_source = (1ll << k) - 1;
  if (n_sources) *n_sources = 1ll << k;
  return TSM_OK;
}

int tsm_binstore_put(tsm_binstore* st, int k, const double* block_sum_host) {
  if (!st || !block_sum_host || k < 0 || k >= kMaxBlocks)
    return fail(TSM_ERR_INVALID_ARG, "tsm_binstore_put: bad argument");
  BlockHeader h;
  memcpy(h.magic, kMagic, 8);
  h.header_bytes = sizeof(h);
  h.k = (uint32_t)k;
  h.first_source = (1ull << k) - 1;
  h.n_sources = 1ull << k;
  h.n_values = st->n_values;
  h.checksum = fnv1a(block_sum_host, st->n_values * sizeof(double));
  const std::string path = block_path(st->prefix, k), tmp = path + ".part";
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return fail(TSM_ERR_INVALID_ARG, "cannot write %s: %s", tmp.c_str(), strerror(errno));
  bool ok = fwrite(&h, 1, sizeof(h), f) == sizeof(h) &&
            fwrite(block_sum_host, sizeof(double), st->n_values, f) == st->n_values;
  ok = (fflush(f) == 0) && ok;
  ok = (fclose(f) == 0) && ok;
  if (!ok || rename(tmp.c_str(), path.c_str()) != 0) {
    remove(tmp.c_str());
    return fail(TSM_ERR_INVALID_ARG, "writing %s failed: %s", path.c_str(), strerror(errno));
  }
  st->present[k] = true;
  return TSM_OK;
}

int tsm_binstore_mean(const tsm_binstore* st, long long n, double* out_host) {
  if (!st || !out_host || n < 1) return fail(TSM_ERR_INVALID_ARG, "tsm_binstore_mean: bad argument");
  std::vector<double> blk(st->n_values);
  for (size_t i = 0; i < st->n_values; ++i) out_host[i] = 0.0;
  for (int k = 0; k < kMaxBlocks && (n >> k); ++k) {
    if (!((n >> k) & 1)) continue;
    if (!st->present[k]) return fail(TSM_ERR_INVALID_ARG, "%lld sources need block %d, which is not stored", n, k);
    TSM_TRY(read_block(st, k, blk.data()));
    for (size_t i = 0; i < st->n_values; ++i) out_host[i] += blk[i];
  }
  for (size_t i = 0; i < st->n_values; ++i) out_host[i] /= (double)n;
  return TSM_OK;
}

int tsm_accumulate_blocks(tsm_gauge* g, const tsm_params* p, tsm_binstore* st, int k_end, tsm_stats* stats,
                          void* stream) {
  if (!g || !p || !st || k_end < 0 || k_end > kMaxBlocks || p->n_mom < 1 || !p->mom)
    return fail(TSM_ERR_INVALID_ARG, "tsm_accumulate_blocks: bad argument");
  if (solver_kind(p->lp_solver) < 0) return fail(TSM_ERR_INVALID_ARG, "bad solver");
  if ((p->lp_solver & TSM_SOLVER_EO) && !eo_lattice(g->geom))
    return fail(TSM_ERR_INVALID_ARG, "even-odd needs even extents in all four directions");
  const unsigned need = solver_link_precs(p->lp_solver);
  if ((g->precisions & need) != need) return fail(TSM_ERR_INVALID_ARG, "solver needs gauge copies 0x%x", need);
  if (!(p->rho_lp > 0 && p->rho_lp < 1) || p->max_iter < 1 || !(p->kappa > 0) || !isfinite(p->mu))
    return fail(TSM_ERR_INVALID_ARG, "bad rho_lp/max_iter/kappa/mu");
  TSM_CUDA(cudaSetDevice(g->ctx->device));
  return accumulate_blocks(g, p, st, k_end, stats, pick_stream(g, stream));
}

}  // extern "C"
